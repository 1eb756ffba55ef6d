"""he_mul_rescale_static (workspace in the library's fixed device scratch)
against he_mul_rescale with a caller-allocated workspace.

Both compute the same modular integer result, so the bar is bit-exactness.
Two calls in a row at different levels and on different inputs check that
the second call does not depend on what the first left in the scratch.
"""
import numpy as np
import pytest

import seeded_inputs as si

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    from paper_2003_04510_gb300 import build
    build.build()
    import paper_2003_04510_gb300 as pkg
    return pkg


def rand_ct(ctx, level, seed):
    q = [int(x) for x in ctx.q[:level]]
    return np.stack([si.uniform_residues(q, (ctx.N,), seed), si.uniform_residues(q, (ctx.N,), seed + 1)])


def rand_evk(ctx, seed):
    ext = [int(x) for x in ctx.moduli]
    return np.stack([np.stack([si.uniform_residues(ext, (ctx.N,), seed + 2 * j),
                               si.uniform_residues(ext, (ctx.N,), seed + 2 * j + 1)]) for j in range(ctx.dnum)])


def both(g, ctx, ct1, ct2, evk_t, level):
    import torch
    a, b = g.to_device(ct1), g.to_device(ct2)
    ref = torch.empty((2, level - 1, ctx.N), dtype=torch.int64, device="cuda")
    g.he_mul_rescale(ctx, a, b, evk_t, level, ref, g.workspace(ctx, level))
    got = torch.full((2, level - 1, ctx.N), -1, dtype=torch.int64, device="cuda")
    g.he_mul_rescale_static(ctx, a, b, evk_t, level, got)
    torch.cuda.synchronize()
    return g.to_host(ref), g.to_host(got)


@pytest.mark.parametrize("name,levels", [("n12", (3, 2)), ("n15", (16, 9))])
def test_static_matches_workspace_entry_point(g, name, levels):
    ctx = g.Context(g.PRESETS[name][0], device=True)
    evk_t = g.to_device(rand_evk(ctx, 500))
    for k, level in enumerate(levels):
        assert g.he_workspace_bytes(ctx, level) <= g.HE_STATIC_SCRATCH_BYTES
        ct1, ct2 = rand_ct(ctx, level, 510 + 10 * k), rand_ct(ctx, level, 520 + 10 * k)
        ref, got = both(g, ctx, ct1, ct2, evk_t, level)
        assert np.array_equal(got, ref), (name, level)


def test_static_rejects_levels_beyond_scratch(g):
    import torch
    ctx = g.Context(g.PRESETS["n16"][0], device=True)
    fits = max(l for l in range(2, ctx.prm.L + 1) if g.he_workspace_bytes(ctx, l) <= g.HE_STATIC_SCRATCH_BYTES)
    assert g.he_workspace_bytes(ctx, fits + 1) > g.HE_STATIC_SCRATCH_BYTES
    a = torch.zeros((2, fits + 1, ctx.N), dtype=torch.int64, device="cuda")
    out = torch.zeros((2, fits, ctx.N), dtype=torch.int64, device="cuda")
    with pytest.raises(g.HeError) as e:
        g.he_mul_rescale_static(ctx, a, a, a, fits + 1, out)
    assert e.value.code == g.HE_ENOMEM
    # the largest level that fits still runs, and matches the workspace entry point
    evk_t = g.to_device(rand_evk(ctx, 530))
    ref, got = both(g, ctx, rand_ct(ctx, fits, 540), rand_ct(ctx, fits, 550), evk_t, fits)
    assert np.array_equal(got, ref)


def test_static_back_to_back_on_one_stream(g):
    """Calls issued in order on one non-default stream share the scratch
    safely: two calls back to back at different levels and on different
    inputs, synchronised only at the end, each equal the workspace entry
    point's result.  A level below 2 is rejected before anything runs."""
    import torch
    ctx = g.Context(g.PRESETS["n15"][0], device=True)
    evk_t = g.to_device(rand_evk(ctx, 560))
    st = torch.cuda.Stream()
    cases = []
    for k, level in enumerate((16, 7)):
        a = g.to_device(rand_ct(ctx, level, 570 + 10 * k))
        b = g.to_device(rand_ct(ctx, level, 575 + 10 * k))
        cases.append((level, a, b, torch.full((2, level - 1, ctx.N), -1, dtype=torch.int64, device="cuda")))
    torch.cuda.synchronize()
    for level, a, b, out in cases:
        g.he_mul_rescale_static(ctx, a, b, evk_t, level, out, st)
    st.synchronize()
    for level, a, b, out in cases:
        ref = torch.empty_like(out)
        g.he_mul_rescale(ctx, a, b, evk_t, level, ref, g.workspace(ctx, level))
        torch.cuda.synchronize()
        assert torch.equal(out, ref), level
    level, a, b, out = cases[0]
    with pytest.raises(g.HeError) as e:
        g.he_mul_rescale_static(ctx, a, b, evk_t, 1, out, st)
    assert e.value.code == g.HE_ELEVEL
