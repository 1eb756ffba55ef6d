"""Pins for the oracle's scheme steps: tensor product, ModUp, inner product /
evaluation key, ModDown, rescale, key generation, encoding and the decryption
bound of the whole HE Mul.

Expected values come from Python big integers: CRT reconstruction, floors of
exact rationals and schoolbook negacyclic products.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import seeded_inputs as si
from oracle.encoding import decode, encode, encode_float

# A tiny parameter set with several digits, a short last digit and several
# special primes: N=16, 5 ciphertext limbs, 3 specials, 2 limbs per digit.
TINY = dict(logN=4, L=5, K=3, alpha=2, q_bits=50, p_bits=52, h=4)


def tiny():
    return oracle.make_params(**TINY)


def crt(res, moduli):
    """Exact CRT value in [0, prod) of one coefficient."""
    M = 1
    for m in moduli:
        M *= m
    v = 0
    for r, m in zip(res, moduli):
        Mh = M // m
        v += int(r) * Mh * pow(Mh % m, -1, m)
    return v % M, M


def to_coeff(prm, X, moduli_psi):
    return np.stack([oracle.intt(X[i], q, psi, prm.logN) for i, (q, psi) in enumerate(moduli_psi)])


def qpsi(prm, l):
    return [(int(prm.q[i]), int(prm.psi_q[i])) for i in range(l)]


def ppsi(prm):
    return [(int(prm.p[k]), int(prm.psi_p[k])) for k in range(prm.K)]


def negacyclic_int(a, b):
    N = len(a)
    c = [0] * N
    for i in range(N):
        for j in range(N):
            if i + j < N:
                c[i + j] += a[i] * b[j]
            else:
                c[i + j - N] -= a[i] * b[j]
    return c


def rand_ct(prm, l, seed):
    rng = np.random.default_rng(seed)
    ct = np.zeros((2, l, prm.N), dtype=np.uint64)
    for h in range(2):
        for i in range(l):
            ct[h, i] = rng.integers(0, int(prm.q[i]), size=prm.N, dtype=np.uint64)
    return ct


def test_tensor_is_ntt_of_negacyclic_products():
    prm, l = tiny(), 4
    ct1, ct2 = rand_ct(prm, l, 1), rand_ct(prm, l, 2)
    d = oracle.tensor(prm, ct1, ct2, l)
    for i, (q, psi) in enumerate(qpsi(prm, l)):
        b1, a1 = (oracle.intt(ct1[h, i], q, psi, prm.logN).tolist() for h in (0, 1))
        b2, a2 = (oracle.intt(ct2[h, i], q, psi, prm.logN).tolist() for h in (0, 1))
        want0 = [x % q for x in negacyclic_int(b1, b2)]
        want1 = [(x + y) % q for x, y in zip(negacyclic_int(a1, b2), negacyclic_int(a2, b1))]
        want2 = [x % q for x in negacyclic_int(a1, a2)]
        for k, want in enumerate([want0, want1, want2]):
            got = oracle.intt(d[k, i], q, psi, prm.logN).tolist()
            assert got == want, (k, i)


@pytest.mark.parametrize("l", [5, 4, 1])
def test_modup_closed_form(l):
    """U_j[t] = X + u * Q_j (mod t), X = CRT_{Q_j}(x), u = floor(sum_i y_i / q_i)."""
    prm = tiny()
    rng = np.random.default_rng(l)
    x = np.stack([rng.integers(0, int(prm.q[i]), size=prm.N, dtype=np.uint64) for i in range(l)])
    ext = prm.ext
    for j in range(prm.beta(l)):
        I = list(prm.digit(j, l))
        qs = [int(prm.q[i]) for i in I]
        U = oracle.modup_digit(prm, x, l, j)
        assert U.shape == (prm.K + l, prm.N)
        for n in range(prm.N):
            X, Qj = crt([x[i, n] for i in I], qs)
            frac = Fraction(0)
            for i, qi in zip(I, qs):
                Qh = Qj // qi
                y = int(x[i, n]) * pow(Qh % qi, -1, qi) % qi
                frac += Fraction(y, qi)
            u = frac.numerator // frac.denominator
            assert 0 <= u < len(I)
            for e in range(prm.K + l):
                t = ext[e]
                if e >= prm.K and (e - prm.K) in I:
                    assert int(U[e, n]) == int(x[e - prm.K, n])
                else:
                    assert int(U[e, n]) == (X + u * Qj) % t


@pytest.mark.parametrize("l", [5, 3])
def test_moddown_closed_form(l):
    """coefficient-domain ModDown output = floor(Y/P) - floor(sum_k y_k/p_k) mod q_i."""
    prm = tiny()
    rng = np.random.default_rng(10 + l)
    ext = prm.ext[: prm.K + l]
    X = np.stack([rng.integers(0, t, size=prm.N, dtype=np.uint64) for t in ext])
    out = oracle.moddown(prm, X, l)
    xc = to_coeff(prm, X, ppsi(prm) + qpsi(prm, l))
    outc = to_coeff(prm, out, qpsi(prm, l))
    ps = [int(v) for v in prm.p]
    P = 1
    for v in ps:
        P *= v
    for n in range(prm.N):
        Y, _ = crt(xc[:, n], ext)
        frac = Fraction(0)
        for k, pk in enumerate(ps):
            Ph = P // pk
            frac += Fraction(int(xc[k, n]) * pow(Ph % pk, -1, pk) % pk, pk)
        v = frac.numerator // frac.denominator
        want = Y // P - v
        for i in range(l):
            qi = int(prm.q[i])
            assert int(outc[i, n]) == want % qi


@pytest.mark.parametrize("l", [5, 2])
def test_rescale_is_exact_floor(l):
    prm = tiny()
    ct = rand_ct(prm, l, 20 + l)
    out = oracle.rescale(prm, ct, l)
    assert out.shape == (2, l - 1, prm.N)
    ql = int(prm.q[l - 1])
    for h in range(2):
        cc = to_coeff(prm, ct[h], qpsi(prm, l))
        oc = to_coeff(prm, out[h], qpsi(prm, l - 1))
        for n in range(prm.N):
            C, _ = crt(cc[:, n], [int(prm.q[i]) for i in range(l)])
            for i in range(l - 1):
                assert int(oc[i, n]) == (C // ql) % int(prm.q[i])


def test_keygen_relations():
    """pk0 - pk1*s and evk_j.b - evk_j.a*s - [i in I_j] P*s^2 are the small Gaussian errors."""
    prm = tiny()
    s = oracle.keygen_sk(prm, 42)
    assert np.count_nonzero(s) == prm.h
    pk = oracle.keygen_pk(prm, s, 42)
    evk = oracle.keygen_evk(prm, s, 42)
    s_int = [int(v) for v in s]
    s2 = negacyclic_int(s_int, s_int)
    P = 1
    for v in prm.p:
        P *= int(v)
    for i, (q, psi) in enumerate(qpsi(prm, prm.L)):
        S = oracle.ntt(np.array([v % q for v in s_int], dtype=np.uint64), q, psi, prm.logN)
        e = oracle.intt(np.array([(int(b) - int(a) * int(sv)) % q for b, a, sv in zip(pk[0, i], pk[1, i], S)],
                                 dtype=np.uint64), q, psi, prm.logN)
        ec = [int(v) if int(v) < q // 2 else int(v) - q for v in e]
        assert max(abs(v) for v in ec) <= 19 and any(ec)
    ext = prm.ext
    for j in range(prm.dnum):
        I = list(prm.digit(j, prm.L))
        errs = []
        for x, t in enumerate(ext):
            psi = int(prm.psi_p[x]) if x < prm.K else int(prm.psi_q[x - prm.K])
            S = oracle.ntt(np.array([v % t for v in s_int], dtype=np.uint64), t, psi, prm.logN)
            diff = [(int(b) - int(a) * int(sv)) % t for b, a, sv in zip(evk[j, 0, x], evk[j, 1, x], S)]
            dc = oracle.intt(np.array(diff, dtype=np.uint64), t, psi, prm.logN).tolist()
            gadget = (x >= prm.K) and (x - prm.K) in I
            if gadget:
                dc = [(v - (P % t) * (c % t)) % t for v, c in zip(dc, s2)]
            ec = [v if v < t // 2 else v - t for v in dc]
            assert max(abs(v) for v in ec) <= 19
            errs.append(ec)
        # the same error polynomial on every limb (it is one integer polynomial)
        assert all(e == errs[0] for e in errs)


@pytest.mark.parametrize("l", [5, 3])
def test_keyswitch_identity_exact(l):
    """KS_b - KS_a*s = P*d2*s^2 + sum_j U_j*e_j (mod P*Q_l), as integer polynomials.

    Pins the evaluation-key gadget, the digit partition, the inner product and
    the NTT-domain bookkeeping of ModUp together."""
    prm = tiny()
    sk = oracle.keygen_sk(prm, 7)
    evk = oracle.keygen_evk(prm, sk, 7)
    rng = np.random.default_rng(30 + l)
    d2 = np.stack([rng.integers(0, int(prm.q[i]), size=prm.N, dtype=np.uint64) for i in range(l)])
    ks, U, KS = oracle.keyswitch(prm, d2, evk, l, want_intermediates=True)
    ext = prm.ext[: prm.K + l]
    mp = ppsi(prm) + qpsi(prm, l)
    M = 1
    for t in ext:
        M *= t
    P = 1
    for v in prm.p:
        P *= int(v)
    s_int = [int(v) for v in sk]
    s2 = negacyclic_int(s_int, s_int)

    def poly(X, moduli):
        xc = to_coeff(prm, X, moduli)
        return [crt(xc[:, n], [m for m, _ in moduli])[0] for n in range(prm.N)]

    KSb, KSa = poly(KS[0], mp), poly(KS[1], mp)
    d2c = poly(d2, qpsi(prm, l))  # only defined mod Q_l; P*d2 is then defined mod P*Q_l
    lhs = [(b - a) % M for b, a in zip(KSb, negacyclic_int(KSa, s_int))]
    rhs = [P * v for v in negacyclic_int(d2c, s2)]
    for j in range(prm.beta(l)):
        e = np.zeros(prm.N, dtype=np.int64)
        oracle.lib().or_sample_gauss(7, 48 + j, prm.sigma, prm.N, oracle._p(e))
        Uj = poly(U[j], mp)
        rhs = [r + v for r, v in zip(rhs, negacyclic_int(Uj, [int(x) for x in e]))]
    assert lhs == [v % M for v in rhs]
    # and ModDown of KS is what the key switch returns
    assert np.array_equal(ks[0], oracle.moddown(prm, KS[0], l))
    assert np.array_equal(ks[1], oracle.moddown(prm, KS[1], l))


def test_encoding_pins():
    logN = 4
    N = 16
    delta = 2.0 ** 30
    z = si.messages(N // 2, 3)
    t = encode_float(z, logN, delta)
    # round trip
    assert np.abs(decode(t / delta, logN) - z).max() < 1e-12
    # a constant message is the constant polynomial
    c = encode_float(np.full(N // 2, 0.75 + 0j), logN, delta)
    assert abs(c[0] - 0.75 * delta) < 1e-3 and np.abs(c[1:]).max() < 1e-3
    # the canonical embedding is a ring homomorphism: slots of t1*t2 are z1*z2
    z2 = si.messages(N // 2, 4)
    t1 = [int(v) for v in encode(z, logN, delta)]
    t2 = [int(v) for v in encode(z2, logN, delta)]
    prod = np.array([float(v) for v in negacyclic_int(t1, t2)]) / delta ** 2
    assert np.abs(decode(prod, logN) - z * z2).max() < 1e-7
    # slot 0 is the evaluation at zeta itself
    zeta = np.exp(1j * np.pi / N)
    assert abs(decode(t / delta, logN)[0] - sum(t[j] / delta * zeta ** j for j in range(N))) < 1e-9


def _fresh(name):
    prm = oracle.preset(name)
    sc = 2.0 ** oracle.PRESETS[name]["scale_bits"]
    ks, s1, s2 = si.SEEDS[name]
    sk = oracle.keygen_sk(prm, ks)
    pk = oracle.keygen_pk(prm, sk, ks)
    m1, m2 = si.messages(prm.N // 2, s1), si.messages(prm.N // 2, s2)
    ct1 = oracle.encrypt_poly(prm, pk, encode(m1, prm.logN, sc), prm.L, s1)
    ct2 = oracle.encrypt_poly(prm, pk, encode(m2, prm.logN, sc), prm.L, s2)
    return prm, sc, sk, pk, m1, m2, ct1, ct2


def test_encrypt_decrypt_fresh_n12():
    prm, sc, sk, pk, m1, m2, ct1, ct2 = _fresh("n12")
    err = np.abs(oracle.decrypt(prm, sk, ct1, prm.L, sc) - m1).max()
    assert 0 < err < 2.0 ** -20
    # a lower level encrypts too (first l limbs of pk)
    ct = oracle.encrypt_poly(prm, pk, encode(m1, prm.logN, sc), 1, 99)
    assert np.abs(oracle.decrypt(prm, sk, ct, 1, sc) - m1).max() < 2.0 ** -20


def test_he_mul_rescale_decrypts_n12():
    """decrypt(rescale(HE Mul(Enc m1, Enc m2))) = m1*m2 within the stated bound (n12: 2^-14)."""
    prm, sc, sk, pk, m1, m2, ct1, ct2 = _fresh("n12")
    evk = oracle.keygen_evk(prm, sk, si.SEEDS["n12"][0])
    c3 = oracle.he_mul(prm, ct1, ct2, evk, prm.L)
    # before rescale: scale Delta^2 at level L
    z3 = oracle.decrypt(prm, sk, c3, prm.L, sc * sc)
    assert np.abs(z3 - m1 * m2).max() < 2.0 ** -20
    c4 = oracle.rescale(prm, c3, prm.L)
    z4 = oracle.decrypt(prm, sk, c4, prm.L - 1, sc * sc / int(prm.q[prm.L - 1]))
    err = np.abs(z4 - m1 * m2).max()
    assert 2.0 ** -40 < err < 2.0 ** -14
    # he_mul is tensor + key switch + add, composed
    d = oracle.tensor(prm, ct1, ct2, prm.L)
    ks = oracle.keyswitch(prm, d[2], evk, prm.L)
    for i in range(prm.L):
        q = int(prm.q[i])
        assert np.array_equal(c3[0, i], (d[0, i] + ks[0, i]) % np.uint64(q))
        assert np.array_equal(c3[1, i], (d[1, i] + ks[1, i]) % np.uint64(q))
