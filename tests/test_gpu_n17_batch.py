"""Batched and served HE Mul at N = 2^17 (44 limbs, 12 special primes, digits
of 11 limbs with a short last digit): every batch entry and every served
request equals the request run alone, and batch entries match the oracle.
"""
import numpy as np
import pytest

import oracle

from test_gpu_parity import ctx_for, dev, g, gpu_mul, host, rand_ct, rand_evk  # noqa: F401

pytestmark = pytest.mark.gpu


def test_batch_n17_matches_single_and_oracle(g):
    import torch
    op = oracle.preset("n17")
    ctx = ctx_for(g, "n17")
    evk = rand_evk(op, 1700)
    evk_t = dev(g, evk)
    levels = [44, 13, 2, 30, 12]
    jobs, singles, cts = [], [], []
    for k, lv in enumerate(levels):
        c1, c2 = rand_ct(op, lv, 1710 + 4 * k), rand_ct(op, lv, 1712 + 4 * k)
        cts.append((c1, c2))
        out = torch.full((2, lv - 1, op.N), -1, dtype=torch.int64, device="cuda")
        jobs.append((dev(g, c1), dev(g, c2), out, lv))
        singles.append(gpu_mul(g, ctx, c1, c2, evk_t, lv, fused=True))
    ws = torch.empty(g.he_batch_workspace_bytes(ctx, levels) // 8, dtype=torch.int64, device="cuda")
    g.he_mul_batch(ctx, jobs, evk_t, ws)
    torch.cuda.synchronize()
    for (_, _, out, lv), single in zip(jobs, singles):
        assert np.array_equal(host(g, out), single), lv
    for k in (1, 2):  # levels 13 (two digits, short second) and 2 (one short digit)
        c1, c2 = cts[k]
        lv = levels[k]
        assert np.array_equal(host(g, jobs[k][2]), oracle.rescale(op, oracle.he_mul(op, c1, c2, evk, lv), lv)), lv


def test_server_n16_n17_mix_matches_single(g):
    import torch
    rings = ["n16", "n17"]
    ctxs = [ctx_for(g, r) for r in rings]
    ops = [oracle.preset(r) for r in rings]
    evks = [dev(g, rand_evk(op, 1800 + i)) for i, op in enumerate(ops)]
    budget = 3 * g.he_batch_workspace_bytes(ctxs[1], [44])
    srv = g.Server(ctxs, evks, hbm_budget=budget, max_batch=4, streams=2)
    rng = np.random.default_rng(17)
    staged = []
    for k in range(12):
        ri = int(rng.random() < 0.5)
        op = ops[ri]
        lv = int(rng.integers(2, op.L + 1))
        c1, c2 = rand_ct(op, lv, 1810 + 2 * k), rand_ct(op, lv, 1830 + 2 * k)
        out = torch.full((2, lv - 1, op.N), -1, dtype=torch.int64, device="cuda")
        staged.append((ri, lv, dev(g, c1), dev(g, c2), out))
    torch.cuda.synchronize()
    reqs = [(ri, lv, t1, t2, out, srv.submit(ri, lv, t1, t2, out)) for ri, lv, t1, t2, out in staged]
    for *_, tk in reqs:
        srv.wait(tk, 120000)
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["pending"] == 0
    srv.close()
    for ri, lv, t1, t2, out, _ in reqs:
        ctx = ctxs[ri]
        alone = torch.empty_like(out)
        g.he_mul_rescale(ctx, t1, t2, evks[ri], lv, alone, g.workspace(ctx, lv))
        torch.cuda.synchronize()
        assert torch.equal(out, alone), (ri, lv)
