"""Pins for the oracle's NTT (Algo 3 / Algo 4) and iNTT.

Expected values: direct evaluation of the polynomial at the odd powers of psi,
schoolbook negacyclic convolution and the operation count of Table 4, all
computed with Python integers.
"""
import random

import numpy as np
import pytest

import oracle

L = oracle.lib()


def bitrev(x, bits):
    r = 0
    for _ in range(bits):
        r = (r << 1) | (x & 1)
        x >>= 1
    return r


def negacyclic(a, b, q):
    N = len(a)
    c = [0] * N
    for i in range(N):
        for j in range(N):
            k = i + j
            if k < N:
                c[k] += a[i] * b[j]
            else:
                c[k - N] -= a[i] * b[j]
    return [x % q for x in c]


def small_prime(logN, bits):
    prm = oracle.make_params(logN, 1, 1, 1, bits, bits + 1)
    return int(prm.q[0]), int(prm.psi_q[0])


CASES = [(97, 4), (7681, 8)] + [small_prime(lg, b) + (lg,) for lg, b in [(3, 50), (4, 54), (6, 55), (5, 62)]]


@pytest.mark.parametrize("case", CASES)
def test_ntt_direct_evaluation(case):
    if len(case) == 2:
        q, logN = case
        psi = L.or_min_psi(q, logN)
    else:
        q, psi, logN = case
    N = 1 << logN
    rng = random.Random(q)
    a = [rng.randrange(q) for _ in range(N)]
    A = oracle.ntt(np.array(a, dtype=np.uint64), q, psi, logN).tolist()
    for i in range(N):
        e = 2 * bitrev(i, logN) + 1
        want = sum(a[k] * pow(psi, e * k, q) for k in range(N)) % q
        assert A[i] == want


@pytest.mark.parametrize("logN,bits", [(3, 50), (5, 54), (6, 55)])
def test_negacyclic_convolution(logN, bits):
    q, psi = small_prime(logN, bits)
    N = 1 << logN
    rng = random.Random(logN)
    a = [rng.randrange(q) for _ in range(N)]
    b = [rng.randrange(q) for _ in range(N)]
    A = oracle.ntt(np.array(a, dtype=np.uint64), q, psi, logN)
    B = oracle.ntt(np.array(b, dtype=np.uint64), q, psi, logN)
    C = np.array([(int(x) * int(y)) % q for x, y in zip(A, B)], dtype=np.uint64)
    c = oracle.intt(C, q, psi, logN).tolist()
    assert c == negacyclic(a, b, q)


@pytest.mark.parametrize("name", ["n12", "n16"])
def test_intt_inverts_ntt_and_op_count(name):
    prm = oracle.preset(name)
    N, logN = prm.N, prm.logN
    rng = np.random.default_rng(5)
    for q, psi in [(int(prm.q[0]), int(prm.psi_q[0])), (int(prm.p[-1]), int(prm.psi_p[-1]))]:
        a = rng.integers(0, q, size=N, dtype=np.uint64)
        a[:3] = [0, 1, q - 1]
        L.or_reset_butterfly_count()
        A = oracle.ntt(a, q, psi, logN)
        assert L.or_butterfly_count() == N // 2 * logN  # Table 4: np * N/2 * log N per prime
        L.or_reset_butterfly_count()
        b = oracle.intt(A, q, psi, logN)
        assert L.or_butterfly_count() == N // 2 * logN
        assert np.array_equal(a, b)
        assert int(A.max()) < q


def test_ntt_of_delta_and_constant():
    # NTT of X^0 is all ones; NTT of the constant c is c everywhere
    q, psi = small_prime(6, 54)
    N = 64
    one = np.zeros(N, dtype=np.uint64)
    one[0] = 7
    assert (oracle.ntt(one, q, psi, 6) == 7).all()
    # NTT of X: slot i holds psi^(2 bitrev(i) + 1)
    x = np.zeros(N, dtype=np.uint64)
    x[1] = 1
    X = oracle.ntt(x, q, psi, 6).tolist()
    assert X == [pow(psi, 2 * bitrev(i, 6) + 1, q) for i in range(N)]
