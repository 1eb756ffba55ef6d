"""GPU parity of the paper's own non-RNS HE Mul (BigInt coefficients modulo
powers of two, CRT / NTT / iCRT products) against the oracle, word for word.
"""
import numpy as np
import pytest

import oracle
import seeded_inputs as si
from oracle.encoding import encode

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    from paper_2003_04510_gb300 import build
    build.build()
    import paper_2003_04510_gb300 as pkg
    return pkg


def nr_context(g, logN, np2):
    return g.Context(g.Params(logN, np2, 1, 16, 57, 57, 64), device=True)


def rand_words(k, N, seed):
    rng = np.random.default_rng(seed)
    a = rng.integers(0, 1 << 63, size=(oracle.nwords(k), N), dtype=np.uint64) * np.uint64(2) + \
        rng.integers(0, 2, size=(oracle.nwords(k), N), dtype=np.uint64)
    if k % 64:
        a[-1] &= np.uint64((1 << (k % 64)) - 1)
    return a


def test_real_keys_small_ring(g):
    """N = 2^12, log Q = 300, log p = 30: encrypt with the oracle, HE Mul and rescale on the GPU."""
    import torch
    prm = oracle.nr_params(12, 300, 30)
    ctx = nr_context(g, 12, prm.np2)
    plan = g.NrPlan(ctx, prm.logQ, prm.logp)
    assert (plan.np1, plan.np2) == (prm.np1, prm.np2)
    assert np.array_equal(ctx.q[: prm.np2], prm.primes)
    sk = oracle.keygen_sk(oracle.make_params(12, 1, 1, 1, 50, 51, h=64), 1212)
    pk, evk = oracle.nr_keygen(prm, sk, 1212)
    sc = 2.0 ** prm.logp
    m1, m2 = si.messages(prm.N // 2, 1213), si.messages(prm.N // 2, 1214)
    c1 = oracle.nr_encrypt(prm, pk, encode(m1, prm.logN, sc), prm.logQ, 1215)
    c2 = oracle.nr_encrypt(prm, pk, encode(m2, prm.logN, sc), prm.logQ, 1216)
    prep = plan.prepare_evk(g.to_device(evk))
    ws = plan.workspace()
    logq = prm.logQ
    out = torch.empty((2, oracle.nwords(logq), prm.N), dtype=torch.int64, device="cuda")
    plan.mul(g.to_device(c1), g.to_device(c2), prep, logq, out, ws)
    torch.cuda.synchronize()
    want = oracle.nr_he_mul(prm, c1, c2, evk, logq)
    got = g.to_host(out)
    assert np.array_equal(got, want)
    rs = torch.empty((2, oracle.nwords(logq - prm.logp), prm.N), dtype=torch.int64, device="cuda")
    plan.rescale(out, logq, rs)
    torch.cuda.synchronize()
    want_rs = oracle.nr_rescale(prm, want, logq)
    assert np.array_equal(g.to_host(rs), want_rs)
    z = oracle.nr_decrypt(prm, sk, want_rs, logq - prm.logp, sc)
    assert np.abs(z - m1 * m2).max() < 2.0 ** -12
    # a lower level: random ciphertexts at log q = 250 (not a multiple of 64)
    logq = 250
    a, b = np.stack([rand_words(logq, prm.N, 1)] * 1 + [rand_words(logq, prm.N, 2)]), \
        np.stack([rand_words(logq, prm.N, 3), rand_words(logq, prm.N, 4)])
    out = torch.empty((2, oracle.nwords(logq), prm.N), dtype=torch.int64, device="cuda")
    plan.mul(g.to_device(a), g.to_device(b), prep, logq, out, ws)
    torch.cuda.synchronize()
    assert np.array_equal(g.to_host(out), oracle.nr_he_mul(prm, a, b, evk, logq))
    plan.close()


@pytest.mark.slow
def test_paper_parameters_n16_logQ1200(g):
    """The paper's workload: N = 2^16, log Q = 1200 (np 43 / 64), random words."""
    import torch
    prm = oracle.nr_params(16, 1200, 30)
    ctx = nr_context(g, 16, prm.np2)
    plan = g.NrPlan(ctx, prm.logQ, prm.logp)
    assert (plan.np1, plan.np2) == (43, 64)
    logq = prm.logQ
    c1 = np.stack([rand_words(logq, prm.N, 11), rand_words(logq, prm.N, 12)])
    c2 = np.stack([rand_words(logq, prm.N, 13), rand_words(logq, prm.N, 14)])
    evk = np.stack([rand_words(2 * prm.logQ, prm.N, 15), rand_words(2 * prm.logQ, prm.N, 16)])
    prep = plan.prepare_evk(g.to_device(evk))
    ws = plan.workspace()
    out = torch.empty((2, oracle.nwords(logq), prm.N), dtype=torch.int64, device="cuda")
    plan.mul(g.to_device(c1), g.to_device(c2), prep, logq, out, ws)
    torch.cuda.synchronize()
    assert np.array_equal(g.to_host(out), oracle.nr_he_mul(prm, c1, c2, evk, logq))
    plan.close()


def test_argument_errors(g):
    import torch
    ctx = nr_context(g, 12, 17)
    with pytest.raises(g.HeError) as e:
        g.NrPlan(ctx, 1200, 30)  # too few primes for log Q = 1200
    assert e.value.code == g.HE_EINVAL
    plan = g.NrPlan(ctx, 300, 30)
    x = torch.zeros((2, 5, 4096), dtype=torch.int64, device="cuda")
    with pytest.raises(g.HeError) as e:
        plan.mul(x, x, x, 301, x, plan.workspace())
    assert e.value.code == g.HE_ELEVEL
    with pytest.raises(g.HeError) as e:
        plan.mul(x, x, x, 300, x, plan.workspace()[:10])
    assert e.value.code == g.HE_ENOMEM
    plan.close()
