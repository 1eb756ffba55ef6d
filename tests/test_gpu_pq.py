"""GPU parity of he_mul_rescale_pq (HE Mul with ModDown and rescale as one
division by P q_{l-1}) against the oracle's or_he_mul_rescale_pq, word for
word: real encryptions at n12 and n16, random residues at n15 and n17 (short
last digit), every NTT plan, and decryption of the GPU result.
"""
import numpy as np
import pytest

import oracle

from test_gpu_parity import ctx_for, dev, g, host, rand_ct, rand_evk, real_inputs  # noqa: F401

pytestmark = pytest.mark.gpu


def gpu_pq(g, ctx, c1, c2, evk_t, level):
    import torch
    out = torch.empty((2, level - 1, ctx.N), dtype=torch.int64, device="cuda")
    g.he_mul_rescale_pq(ctx, dev(g, c1), dev(g, c2), evk_t, level, out, g.workspace(ctx, level))
    torch.cuda.synchronize()
    return host(g, out)


def cut(ct, level):
    return np.ascontiguousarray(np.stack([ct[0, :level], ct[1, :level]]))


def test_pq_n12_every_level_and_decrypts(g):
    op, sc, sk, pk, evk, m1, m2, ct1, ct2 = real_inputs("n12")
    ctx = ctx_for(g, "n12")
    evk_t = dev(g, evk)
    for level in (3, 2):
        c1, c2 = cut(ct1, level), cut(ct2, level)
        got = gpu_pq(g, ctx, c1, c2, evk_t, level)
        assert np.array_equal(got, oracle.he_mul_rescale_pq(op, c1, c2, evk, level)), level
    z = oracle.decrypt(op, sk, got, 1, sc * sc / int(op.q[1]))
    assert np.abs(z - m1 * m2).max() < 2.0 ** -14


@pytest.mark.parametrize("level", [24, 9])
def test_pq_n16_real_keys(g, level):
    op, sc, sk, pk, evk, m1, m2, ct1, ct2 = real_inputs("n16")
    ctx = ctx_for(g, "n16")
    evk_t = dev(g, evk)
    c1, c2 = cut(ct1, level), cut(ct2, level)
    want = oracle.he_mul_rescale_pq(op, c1, c2, evk, level)
    try:
        for shape in ((1, 8, 1, 0), (2, 16, 1, 15), (1, 8, 2, 15, 8, 7, 1, 1)):
            g.he_set_shape(ctx, *shape)
            assert np.array_equal(gpu_pq(g, ctx, c1, c2, evk_t, level), want), shape
    finally:
        g.he_set_shape(ctx, 4, 8, 1)
    # The conversion's overflow term u < K + 1 is not divided by q_{l-1} here
    # (after a separate ModDown it is), so the additive error per coefficient
    # is up to K + 2 instead of 1: the two-floor bound 2^-24 times K + 2 = 10.
    z = oracle.decrypt(op, sk, want, level - 1, sc * sc / int(op.q[level - 1]))
    err = np.abs(z - m1 * m2).max()
    assert 2.0 ** -40 < err < (op.K + 2) * 2.0 ** -24


@pytest.mark.parametrize("name,level", [("n15", 16), ("n15", 2), ("n17", 13)])
def test_pq_random_residues(g, name, level):
    op = oracle.preset(name)
    ctx = ctx_for(g, name)
    evk = rand_evk(op, 1300 + level)
    c1, c2 = rand_ct(op, level, 1310 + level), rand_ct(op, level, 1320 + level)
    got = gpu_pq(g, ctx, c1, c2, dev(g, evk), level)
    assert np.array_equal(got, oracle.he_mul_rescale_pq(op, c1, c2, evk, level))
    # and it is not the two-floor result
    assert not np.array_equal(got, oracle.rescale(op, oracle.he_mul(op, c1, c2, evk, level), level))


def test_pq_argument_errors(g):
    import torch
    op = oracle.preset("n12")
    ctx = ctx_for(g, "n12")
    evk_t = dev(g, rand_evk(op, 1400))
    a = dev(g, rand_ct(op, 3, 1401))
    out = torch.empty((2, 2, op.N), dtype=torch.int64, device="cuda")
    ws = g.workspace(ctx, 3)
    for level, code in ((1, g.HE_ELEVEL), (4, g.HE_ELEVEL)):
        with pytest.raises(g.HeError) as e:
            g.he_mul_rescale_pq(ctx, a, a, evk_t, level, out, ws)
        assert e.value.code == code
    with pytest.raises(g.HeError) as e:
        g.he_mul_rescale_pq(ctx, a, a, evk_t, 3, out, ws[: ws.numel() // 2])
    assert e.value.code == g.HE_ENOMEM
