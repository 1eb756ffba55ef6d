"""Pins for the oracle's rotation (Galois automorphism + key switching).

HE rotation is not in the paper; it reuses the paper's key switching (Fig. 2,
region 2) with a key for kappa_g(s).  The automorphism is pinned by evaluating
polynomials at roots of unity and by polynomial substitution with Python
integers, the rotation key by its defining relation, and the whole rotation by
the key-switching identity and by decryption (slots rotated / conjugated).
"""
import numpy as np
import pytest

import oracle
import seeded_inputs as si
from oracle.encoding import encode

from test_oracle_scheme import TINY, crt, negacyclic_int, ppsi, qpsi, tiny, to_coeff


def _root(q, N):
    """A primitive 2N-th root of unity mod q (q = 1 mod 2N prime)."""
    for x in range(2, q):
        r = pow(x, (q - 1) // (2 * N), q)
        if pow(r, N, q) == q - 1:
            return r
    raise AssertionError


def _eval(a, x, q):
    v = 0
    for c in reversed([int(t) for t in a]):
        v = (v * x + c) % q
    return v


@pytest.mark.parametrize("N,q", [(16, 97), (32, 193), (64, 257)])
def test_automorphism_evaluation(N, q):
    """kappa_g(a)(w^e) = a(w^(g e)) at every primitive 2N-th root w^e (e odd)."""
    logN = N.bit_length() - 1
    w = _root(q, N)
    rng = np.random.default_rng(N)
    a = rng.integers(0, q, size=N, dtype=np.uint64)
    for g in (1, 3, 5, 25 % (2 * N), 2 * N - 1, 2 * N - 5):
        ka = oracle.automorphism(a, q, g, logN)
        for e in range(1, 2 * N, 2):
            assert _eval(ka, pow(w, e, q), q) == _eval(a, pow(w, g * e % (2 * N), q), q), (g, e)


def test_automorphism_substitution_and_group():
    """a(X^g) by schoolbook substitution; kappa_g kappa_h = kappa_gh; multiplicative."""
    N, logN, q = 16, 4, 97
    rng = np.random.default_rng(4)
    a = [int(v) for v in rng.integers(0, q, size=N)]
    b = [int(v) for v in rng.integers(0, q, size=N)]
    for g in (3, 5, 31, 13):
        # X^g as a polynomial, then sum_i a_i (X^g)^i with negacyclic products
        xg = [0] * N
        xg[g % N] = 1 if (g // N) % 2 == 0 else -1
        acc, power = [0] * N, [1] + [0] * (N - 1)
        for i in range(N):
            acc = [u + a[i] * v for u, v in zip(acc, power)]
            power = negacyclic_int(power, xg)
        want = [v % q for v in acc]
        assert oracle.automorphism(np.array(a, dtype=np.uint64), q, g, logN).tolist() == want
    A = np.array(a, dtype=np.uint64)
    for g, h in ((3, 5), (5, 5), (31, 7)):
        gh = g * h % (2 * N)
        assert np.array_equal(oracle.automorphism(oracle.automorphism(A, q, h, logN), q, g, logN),
                              oracle.automorphism(A, q, gh, logN))
    assert np.array_equal(oracle.automorphism(A, q, 1, logN), A)
    ab = [v % q for v in negacyclic_int(a, b)]
    kab = oracle.automorphism(np.array(ab, dtype=np.uint64), q, 5, logN).tolist()
    ka = [int(v) for v in oracle.automorphism(A, q, 5, logN)]
    kb = [int(v) for v in oracle.automorphism(np.array(b, dtype=np.uint64), q, 5, logN)]
    assert kab == [v % q for v in negacyclic_int(ka, kb)]


def test_automorphism_is_a_permutation_in_the_ntt_domain():
    """NTT(kappa_g(a))[i] = NTT(a)[j] with 2 br(j) + 1 = g (2 br(i) + 1) mod 2N."""
    prm = oracle.preset("n12")
    N, logN = prm.N, prm.logN
    br = [int(format(i, f"0{logN}b")[::-1], 2) for i in range(N)]
    q, psi = int(prm.q[0]), int(prm.psi_q[0])
    rng = np.random.default_rng(12)
    a = rng.integers(0, q, size=N, dtype=np.uint64)
    A = oracle.ntt(a, q, psi, logN)
    for g in (oracle.galois_elt(prm, 1), oracle.galois_elt(prm, -3), oracle.conj_elt(prm)):
        KA = oracle.ntt(oracle.automorphism(a, q, g, logN), q, psi, logN)
        src = [br[((g * (2 * br[i] + 1)) % (2 * N) - 1) // 2] for i in range(N)]
        assert np.array_equal(KA, A[src]), g


def test_rotation_key_relation():
    """rk_j.b - rk_j.a*s - [i in I_j] P*kappa_g(s) is one small error polynomial."""
    prm = tiny()
    s = oracle.keygen_sk(prm, 11)
    g = oracle.galois_elt(prm, 1)
    rk = oracle.keygen_rot(prm, s, g, 11)
    s_int = [int(v) for v in s]
    ks = [0] * prm.N
    for i, v in enumerate(s_int):
        e = i * g % (2 * prm.N)
        if e < prm.N:
            ks[e] += v
        else:
            ks[e - prm.N] -= v
    P = 1
    for v in prm.p:
        P *= int(v)
    for j in range(prm.dnum):
        I = list(prm.digit(j, prm.L))
        errs = []
        for x, t in enumerate(prm.ext):
            psi = int(prm.psi_p[x]) if x < prm.K else int(prm.psi_q[x - prm.K])
            S = oracle.ntt(np.array([v % t for v in s_int], dtype=np.uint64), t, psi, prm.logN)
            diff = [(int(b) - int(a) * int(sv)) % t for b, a, sv in zip(rk[j, 0, x], rk[j, 1, x], S)]
            dc = oracle.intt(np.array(diff, dtype=np.uint64), t, psi, prm.logN).tolist()
            if x >= prm.K and (x - prm.K) in I:
                dc = [(v - (P % t) * (c % t)) % t for v, c in zip(dc, ks)]
            ec = [v if v < t // 2 else v - t for v in dc]
            assert max(abs(v) for v in ec) <= 19
            errs.append(ec)
        assert all(e == errs[0] for e in errs) and any(errs[0])
    # a different Galois element gives a different key (kappa_g(s) changes)
    assert not np.array_equal(rk, oracle.keygen_rot(prm, s, oracle.galois_elt(prm, 2), 11))


@pytest.mark.parametrize("l", [5, 2])
def test_rotate_is_automorphism_then_keyswitch(l):
    """rotate = (kappa(b) + ks_b, ks_a) with ks = keyswitch(-kappa(a), rk), and
    out.b - out.a*s = kappa(b) - kappa(a)*kappa(s) + ModDown noise (integer check)."""
    prm = tiny()
    sk = oracle.keygen_sk(prm, 21)
    g = oracle.galois_elt(prm, 3)
    rk = oracle.keygen_rot(prm, sk, g, 21)
    rng = np.random.default_rng(40 + l)
    ct = np.stack([np.stack([rng.integers(0, int(prm.q[i]), size=prm.N, dtype=np.uint64) for i in range(l)])
                   for _ in range(2)])
    out = oracle.rotate(prm, ct, g, rk, l)
    kap = np.zeros_like(ct)
    for h in range(2):
        for i, (q, psi) in enumerate(qpsi(prm, l)):
            c = oracle.intt(ct[h, i], q, psi, prm.logN)
            kap[h, i] = oracle.ntt(oracle.automorphism(c, q, g, prm.logN), q, psi, prm.logN)
    x = np.stack([(np.uint64(int(prm.q[i])) - kap[1, i]) % np.uint64(int(prm.q[i])) for i in range(l)])
    ks = oracle.keyswitch(prm, x, rk, l)
    for i in range(l):
        q = np.uint64(int(prm.q[i]))
        assert np.array_equal(out[0, i], (kap[0, i] + ks[0, i]) % q)
        assert np.array_equal(out[1, i], ks[1, i])
    # decryption relation as integers mod Q_l: out.b - out.a s - (kappa(b) - kappa(a) kappa(s)) is small
    s_int = [int(v) for v in sk]
    ksk = oracle.automorphism(np.array([v % int(prm.q[0]) for v in s_int], dtype=np.uint64), int(prm.q[0]), g,
                              prm.logN)
    ksk = [int(v) if int(v) < int(prm.q[0]) // 2 else int(v) - int(prm.q[0]) for v in ksk]
    mq = qpsi(prm, l)
    Q = 1
    for m, _ in mq:
        Q *= m

    def poly(X):
        xc = to_coeff(prm, X, mq)
        return [crt(xc[:, n], [m for m, _ in mq])[0] for n in range(prm.N)]

    ob, oa, kb, ka = poly(out[0]), poly(out[1]), poly(kap[0]), poly(kap[1])
    lhs = [(b - a) % Q for b, a in zip(ob, negacyclic_int(oa, s_int))]
    rhs = [(b - a) % Q for b, a in zip(kb, negacyclic_int(ka, ksk))]
    diff = [(u - v) % Q for u, v in zip(lhs, rhs)]
    diff = [d if d <= Q // 2 else d - Q for d in diff]
    # key-switching noise: (sum_j U_j e_j)/P + rounding, far below Q_l
    assert max(abs(d) for d in diff) < 2 ** 40


def _fresh_n12():
    prm = oracle.preset("n12")
    sc = 2.0 ** oracle.PRESETS["n12"]["scale_bits"]
    ks, s1, _ = si.SEEDS["n12"]
    sk = oracle.keygen_sk(prm, ks)
    pk = oracle.keygen_pk(prm, sk, ks)
    m = si.messages(prm.N // 2, s1)
    ct = oracle.encrypt_poly(prm, pk, encode(m, prm.logN, sc), prm.L, s1)
    return prm, sc, sk, m, ct


@pytest.mark.parametrize("steps", [1, 5, -1])
def test_rotate_decrypts_to_rotated_slots_n12(steps):
    prm, sc, sk, m, ct = _fresh_n12()
    g = oracle.galois_elt(prm, steps)
    rk = oracle.keygen_rot(prm, sk, g, 1300 + steps % 97)
    out = oracle.rotate(prm, ct, g, rk, prm.L)
    z = oracle.decrypt(prm, sk, out, prm.L, sc)
    err = np.abs(z - np.roll(m, -steps)).max()
    assert 0 < err < 2.0 ** -16, err


def test_conjugate_decrypts_to_conjugate_slots_n12():
    prm, sc, sk, m, ct = _fresh_n12()
    g = oracle.conj_elt(prm)
    rk = oracle.keygen_rot(prm, sk, g, 1399)
    z = oracle.decrypt(prm, sk, oracle.rotate(prm, ct, g, rk, prm.L), prm.L, sc)
    err = np.abs(z - np.conj(m)).max()
    assert 0 < err < 2.0 ** -16, err
