"""Pins for the oracle's word arithmetic, primes, roots and random words.

Every expected value here comes from Python integers, sympy, brute force or a
published vector -- never from the oracle itself.
"""
import os
import random

import numpy as np
import pytest
import sympy

import oracle

L = oracle.lib()


def test_modular_word_ops_against_python_ints():
    rng = random.Random(7)
    moduli = [97, 65537, (1 << 50) - 27, int(oracle.preset("n16").q[0]), int(oracle.preset("n16").p[0]),
              (1 << 62) - 57]
    for q in moduli:
        edges = [0, 1, 2, q - 2, q - 1]
        cases = [(a, b) for a in edges for b in edges] + [(rng.randrange(q), rng.randrange(q)) for _ in range(3000)]
        for a, b in cases:
            assert L.or_mulmod(a, b, q) == (a * b) % q
            assert L.or_addmod(a, b, q) == (a + b) % q
            assert L.or_submod(a, b, q) == (a - b) % q
        for a in [1, 2, q - 1] + [rng.randrange(1, q) for _ in range(50)]:
            e = rng.randrange(1 << 62)
            assert L.or_powmod(a, e, q) == pow(a, e, q)
            if sympy.isprime(q):
                assert (L.or_invmod(a, q) * a) % q == 1


def test_primality_against_sympy():
    rng = random.Random(3)
    # Carmichael numbers and strong pseudoprimes to several small bases
    tricky = [561, 1105, 1729, 2047, 3215031751, 2152302898747, 3474749660383, 341550071728321,
              3825123056546413051, 318665857834031151167461 % (1 << 64)]
    nums = tricky + [rng.randrange(1 << 64) for _ in range(2000)] + list(range(0, 300))
    nums += [int(sympy.prevprime(rng.randrange(1 << 40, 1 << 63))) for _ in range(50)]
    for n in nums:
        assert bool(L.or_is_prime(n)) == sympy.isprime(n), n


@pytest.mark.parametrize("name", ["n12", "n15", "n16", "n17"])
def test_prime_chain_is_the_largest_ntt_friendly_set(name):
    prm = oracle.preset(name)
    twoN = 2 * prm.N
    q = [int(x) for x in prm.q]
    p = [int(x) for x in prm.p]
    assert len(q) == prm.L and len(p) == prm.K
    assert q == sorted(q, reverse=True) and p == sorted(p, reverse=True)
    assert not set(q) & set(p)
    for v in q:
        assert sympy.isprime(v) and v % twoN == 1 and v < (1 << prm.q_bits)
    for v in p:
        assert sympy.isprime(v) and v % twoN == 1 and v < (1 << prm.p_bits)
    # exhaustive: every NTT-friendly prime in [min(q), 2^q_bits) is in the chain
    c = ((1 << prm.q_bits) - 2) // twoN * twoN + 1
    found = []
    while c >= q[-1]:
        if sympy.isprime(c):
            found.append(c)
        c -= twoN
    assert found == q
    # specials: the largest NTT-friendly primes below 2^p_bits that are not ciphertext primes
    c = ((1 << prm.p_bits) - 2) // twoN * twoN + 1
    found = []
    while len(found) < prm.K:
        if sympy.isprime(c) and c not in q:
            found.append(c)
        c -= twoN
    assert found == p


def _all_primitive_roots(q, N):
    # brute force over the whole group for tiny q
    return [x for x in range(1, q) if pow(x, N, q) == q - 1]


@pytest.mark.parametrize("q,logN", [(97, 4), (257, 5), (7681, 8), (12289, 10), (40961, 12)])
def test_min_psi_brute_force_small(q, logN):
    N = 1 << logN
    assert L.or_min_psi(q, logN) == min(_all_primitive_roots(q, N))


@pytest.mark.parametrize("name", ["n12", "n16"])
def test_min_psi_large_primes(name):
    prm = oracle.preset(name)
    N = prm.N
    for q, psi in list(zip(prm.q, prm.psi_q))[:3] + list(zip(prm.p, prm.psi_p))[:2]:
        q, psi = int(q), int(psi)
        assert pow(psi, N, q) == q - 1  # order exactly 2N
        # the primitive 2N-th roots are psi^(2k+1); psi must be the least of them
        g2 = psi * psi % q
        cur, best = psi, psi
        for _ in range(N - 1):
            cur = cur * g2 % q
            best = min(best, cur)
        assert best == psi


def test_splitmix64_published_vectors():
    path = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 6
    for s, i, v in rows:
        assert L.or_splitmix64(int(s), int(i)) == int(v)


def test_samplers_distributions():
    n = 200000
    g = np.zeros(n, dtype=np.int64)
    L.or_sample_gauss(11, 5, 3.2, n, oracle._p(g))
    assert abs(g.mean()) < 0.05 and abs(g.std() - 3.2) < 0.05 and np.abs(g).max() <= 19
    z = np.zeros(n, dtype=np.int64)
    L.or_sample_zo(11, 4, n, oracle._p(z))
    assert set(np.unique(z)) == {-1, 0, 1}
    assert abs((z == 0).mean() - 0.5) < 0.01 and abs((z == 1).mean() - 0.25) < 0.01
    t = (1 << 54) - 33
    u = np.zeros(n, dtype=np.uint64)
    L.or_sample_uniform(11, 2, t, n, oracle._p(u))
    assert int(u.max()) < t and abs(u.astype(np.float64).mean() / t - 0.5) < 0.01
    # HWT secret: exactly h entries of +-1
    prm = oracle.preset("n16")
    s = oracle.keygen_sk(prm, 1601)
    assert np.count_nonzero(s) == prm.h and set(np.unique(s)) == {-1, 0, 1}
    # distinct seeds give distinct secrets; the same seed the same one
    assert not np.array_equal(s, oracle.keygen_sk(prm, 1602))
    assert np.array_equal(s, oracle.keygen_sk(prm, 1601))
