"""GPU parity of the host-buffer entry points: he_mul_rescale_host (one job,
synchronous) and he_mul_rescale_host_stream (a pipelined stream of jobs at
mixed levels, uploads and downloads on their own streams), each result
against the oracle's HE Mul + rescale, word for word.
"""
import numpy as np
import pytest

import oracle

from test_gpu_parity import ctx_for, dev, g, rand_ct, rand_evk  # noqa: F401  (g is a fixture)

pytestmark = pytest.mark.gpu


def pinned(a):
    """A page-locked host copy of a uint64 array (numpy view of a pinned tensor)."""
    import torch
    t = torch.empty(a.size, dtype=torch.int64).pin_memory()
    v = t.numpy().view(np.uint64).reshape(a.shape)
    v[...] = a
    return t, v


def pinned_empty(shape):
    import torch
    t = torch.empty(int(np.prod(shape)), dtype=torch.int64).pin_memory()
    return t, t.numpy().view(np.uint64).reshape(shape)


def want(op, a, b, evk, level):
    return oracle.rescale(op, oracle.he_mul(op, a, b, evk, level), level)


def test_host_call_one_job(g):
    import torch
    op = oracle.preset("n15")
    ctx = ctx_for(g, "n15")
    evk = rand_evk(op, 300)
    evk_t = dev(g, evk)
    for level in (16, 3):
        a, b = rand_ct(op, level, 310 + level), rand_ct(op, level, 320 + level)
        ws = torch.empty(g.he_host_workspace_bytes(ctx, level) // 8, dtype=torch.int64, device="cuda")
        _, pa = pinned(a)
        _, pb = pinned(b)
        _, po = pinned_empty((2, level - 1, op.N))
        g.he_mul_rescale_host(ctx, pa, pb, evk_t, level, po, ws)
        assert np.array_equal(po, want(op, a, b, evk, level)), level


@pytest.mark.parametrize("slots", [2, 3])
def test_host_stream_mixed_levels(g, slots):
    import torch
    op = oracle.preset("n15")
    ctx = ctx_for(g, "n15")
    evk = rand_evk(op, 400)
    evk_t = dev(g, evk)
    levels = [16, 5, 16, 9, 2, 12, 16]
    jobs = [(rand_ct(op, lv, 410 + 4 * k), rand_ct(op, lv, 412 + 4 * k)) for k, lv in enumerate(levels)]
    keep = []
    ct1s, ct2s, outs = [], [], []
    for (a, b), lv in zip(jobs, levels):
        ta, pa = pinned(a)
        tb, pb = pinned(b)
        to, po = pinned_empty((2, lv - 1, op.N))
        keep += [ta, tb, to]
        ct1s.append(pa)
        ct2s.append(pb)
        outs.append(po)
    ws = torch.empty(g.he_host_stream_workspace_bytes(ctx, max(levels), slots) // 8, dtype=torch.int64,
                     device="cuda")
    g.he_mul_rescale_host_stream(ctx, ct1s, ct2s, levels, outs, evk_t, ws, slots=slots)
    for k, ((a, b), lv) in enumerate(zip(jobs, levels)):
        assert np.array_equal(outs[k], want(op, a, b, evk, lv)), (k, lv)


def test_host_stream_pageable_and_repeated_output(g):
    """Pageable host buffers (synchronous copies) and one output buffer
    shared by every job: the last job's result is the one left."""
    import torch
    op = oracle.preset("n12")
    ctx = ctx_for(g, "n12")
    evk = rand_evk(op, 500)
    evk_t = dev(g, evk)
    level = 3
    jobs = [(rand_ct(op, level, 510 + 4 * k), rand_ct(op, level, 512 + 4 * k)) for k in range(5)]
    out = np.zeros((2, level - 1, op.N), dtype=np.uint64)
    ws = torch.empty(g.he_host_stream_workspace_bytes(ctx, level, 2) // 8, dtype=torch.int64, device="cuda")
    g.he_mul_rescale_host_stream(ctx, [a for a, _ in jobs], [b for _, b in jobs], [level] * 5, [out] * 5, evk_t,
                                 ws)
    a, b = jobs[-1]
    assert np.array_equal(out, want(op, a, b, evk, level))


def test_host_stream_argument_errors(g):
    import torch
    op = oracle.preset("n12")
    ctx = ctx_for(g, "n12")
    evk_t = dev(g, rand_evk(op, 600))
    a = rand_ct(op, 3, 610)
    out = np.zeros((2, 2, op.N), dtype=np.uint64)
    assert g.he_host_stream_workspace_bytes(ctx, 3, 1) == 0
    assert g.he_host_stream_workspace_bytes(ctx, 3, 5) == 0
    assert g.he_host_stream_workspace_bytes(ctx, 4, 2) == 0  # above L
    need = g.he_host_stream_workspace_bytes(ctx, 3, 2)
    ws = torch.empty(need // 8, dtype=torch.int64, device="cuda")
    g.he_mul_rescale_host_stream(ctx, [], [], [], [], evk_t, ws)  # nothing to do
    for slots, code in ((1, g.HE_EINVAL), (5, g.HE_EINVAL)):
        with pytest.raises(g.HeError) as e:
            g.he_mul_rescale_host_stream(ctx, [a], [a], [3], [out], evk_t, ws, slots=slots)
        assert e.value.code == code
    with pytest.raises(g.HeError) as e:
        g.he_mul_rescale_host_stream(ctx, [a], [a], [1], [out], evk_t, ws)
    assert e.value.code == g.HE_ELEVEL
    with pytest.raises(g.HeError) as e:
        g.he_mul_rescale_host_stream(ctx, [a], [a], [3], [out], evk_t, ws[: need // 8 - 1])
    assert e.value.code == g.HE_ENOMEM
