"""GPU parity: every CUDA step and the whole HE Mul path, called through the
C ABI, against the CPU oracle on the same seeded inputs.

All arithmetic is modular integer arithmetic, so the bar is bit-exactness:
every output word must equal the oracle's.  Sizes span several NTT tiles and
ragged digit partitions (a short last digit), from N = 2^12 to the full
N = 2^17 configuration.
"""
import numpy as np
import pytest

import oracle
import seeded_inputs as si
from oracle.encoding import encode

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session")
def g():
    from paper_2003_04510_gb300 import build
    build.build()
    import paper_2003_04510_gb300 as pkg
    return pkg


_ctx = {}


def ctx_for(g, name):
    if name not in _ctx:
        _ctx[name] = g.Context(g.PRESETS[name][0], device=True)
    return _ctx[name]


def rand_polys(moduli, N, seed):
    return si.uniform_residues([int(m) for m in moduli], (N,), seed)


def rand_ct(op, level, seed):
    q = [int(x) for x in op.q[:level]]
    return np.stack([rand_polys(q, op.N, seed), rand_polys(q, op.N, seed + 1)])


def rand_evk(op, seed):
    return np.stack([np.stack([rand_polys(op.ext, op.N, seed + 2 * j), rand_polys(op.ext, op.N, seed + 2 * j + 1)])
                     for j in range(op.dnum)])


def dev(g, a):
    return g.to_device(a)


def host(g, t):
    return g.to_host(t)


# ---------------------------------------------------------------------------
# per-step parity
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["n12", "n15", "n16", "n17"])
def test_ntt_forward_inverse_parity(g, name):
    import torch
    ctx = ctx_for(g, name)
    op = oracle.preset(name)
    E = op.K + op.L
    idx = sorted({0, op.K - 1, op.K, E - 1, op.K + op.L // 2})
    mods = [op.ext[e] for e in idx]
    psis = [int(op.psi_p[e]) if e < op.K else int(op.psi_q[e - op.K]) for e in idx]
    a = rand_polys(mods, op.N, 11)
    a[0, :4] = [0, 1, mods[0] - 1, mods[0] - 2]
    a[-1, :] = mods[-1] - 1  # the largest residue everywhere
    want = np.stack([oracle.ntt(a[i], mods[i], psis[i], op.logN) for i in range(len(idx))])
    t = dev(g, a)
    g.he_step_ntt(ctx, t, idx, inverse=False)
    torch.cuda.synchronize()
    assert np.array_equal(host(g, t), want)
    g.he_step_ntt(ctx, t, idx, inverse=True)
    torch.cuda.synchronize()
    assert np.array_equal(host(g, t), a)
    # inverse of fresh data against the oracle's iNTT
    b = rand_polys(mods, op.N, 12)
    want_i = np.stack([oracle.intt(b[i], mods[i], psis[i], op.logN) for i in range(len(idx))])
    t = dev(g, b)
    g.he_step_ntt(ctx, t, idx, inverse=True)
    torch.cuda.synchronize()
    assert np.array_equal(host(g, t), want_i)


@pytest.mark.parametrize("name,level", [("n12", 3), ("n12", 1), ("n16", 24), ("n16", 7)])
def test_tensor_parity(g, name, level):
    import torch
    ctx = ctx_for(g, name)
    op = oracle.preset(name)
    ct1, ct2 = rand_ct(op, level, 21), rand_ct(op, level, 23)
    d = torch.empty((3, level, op.N), dtype=torch.int64, device="cuda")
    g.he_step_tensor(ctx, dev(g, ct1), dev(g, ct2), level, d)
    torch.cuda.synchronize()
    assert np.array_equal(host(g, d), oracle.tensor(op, ct1, ct2, level))


@pytest.mark.parametrize("name,level", [("n12", 3), ("n12", 2), ("n12", 1), ("n16", 24), ("n16", 17), ("n16", 1)])
def test_modup_parity(g, name, level):
    import torch
    ctx = ctx_for(g, name)
    op = oracle.preset(name)
    E, beta = op.K + level, op.beta(level)
    d2 = rand_polys(op.q[:level], op.N, 31)
    U = torch.zeros((beta, E, op.N), dtype=torch.int64, device="cuda")
    ws = g.workspace(ctx, level)
    g.he_step_modup(ctx, dev(g, d2), level, U, ws)
    torch.cuda.synchronize()
    got = host(g, U)
    x = np.stack([oracle.intt(d2[i], int(op.q[i]), int(op.psi_q[i]), op.logN) for i in range(level)])
    for j in range(beta):
        want = oracle.modup_digit(op, x, level, j)
        own = [op.K + i for i in op.digit(j, level)]
        rows = [e for e in range(E) if e not in own]
        assert np.array_equal(got[j, rows], want[rows]), j


@pytest.mark.parametrize("name,level", [("n12", 3), ("n12", 2), ("n16", 24), ("n16", 17)])
def test_inner_product_parity(g, name, level):
    import torch
    ctx = ctx_for(g, name)
    op = oracle.preset(name)
    E, beta = op.K + level, op.beta(level)
    ext = op.ext[:E]
    U = np.stack([rand_polys(ext, op.N, 41 + j) for j in range(beta)])
    d2 = rand_polys(op.q[:level], op.N, 40)
    for j in range(beta):  # the oracle sees d2 in the own-digit rows
        for i in op.digit(j, level):
            U[j, op.K + i] = d2[i]
    evk = rand_evk(op, 50)
    KS = torch.empty((2, E, op.N), dtype=torch.int64, device="cuda")
    g.he_step_inner_product(ctx, dev(g, U), dev(g, d2), dev(g, evk), level, KS, g.workspace(ctx, level))
    torch.cuda.synchronize()
    assert np.array_equal(host(g, KS), oracle.inner_product(op, U, evk, level))


@pytest.mark.parametrize("name,level", [("n12", 3), ("n12", 1), ("n16", 24), ("n16", 5)])
def test_moddown_parity(g, name, level):
    import torch
    ctx = ctx_for(g, name)
    op = oracle.preset(name)
    X = rand_polys(op.ext[: op.K + level], op.N, 61)
    out = torch.empty((level, op.N), dtype=torch.int64, device="cuda")
    g.he_step_moddown(ctx, dev(g, X), level, out, g.workspace(ctx, level))
    torch.cuda.synchronize()
    assert np.array_equal(host(g, out), oracle.moddown(op, X, level))


# ---------------------------------------------------------------------------
# the whole path
# ---------------------------------------------------------------------------
_keys = {}


def real_inputs(name):
    """Oracle-generated keys and ciphertexts (fresh encryptions at level L)."""
    if name not in _keys:
        op = oracle.preset(name)
        sc = 2.0 ** oracle.PRESETS[name]["scale_bits"]
        ks, s1, s2 = si.SEEDS[name]
        sk = oracle.keygen_sk(op, ks)
        pk = oracle.keygen_pk(op, sk, ks)
        evk = oracle.keygen_evk(op, sk, ks)
        m1, m2 = si.messages(op.N // 2, s1), si.messages(op.N // 2, s2)
        ct1 = oracle.encrypt_poly(op, pk, encode(m1, op.logN, sc), op.L, s1)
        ct2 = oracle.encrypt_poly(op, pk, encode(m2, op.logN, sc), op.L, s2)
        _keys[name] = (op, sc, sk, pk, evk, m1, m2, ct1, ct2)
    return _keys[name]


def gpu_mul(g, ctx, ct1, ct2, evk_t, level, fused):
    import torch
    N = ctx.N
    out = torch.empty((2, level - 1 if fused else level, N), dtype=torch.int64, device="cuda")
    ws = g.workspace(ctx, level)
    (g.he_mul_rescale if fused else g.he_mul)(ctx, dev(g, ct1), dev(g, ct2), evk_t, level, out, ws)
    torch.cuda.synchronize()
    return host(g, out)


def test_he_mul_n12_every_level(g):
    import torch
    op, sc, sk, pk, evk, m1, m2, ct1, ct2 = real_inputs("n12")
    ctx = ctx_for(g, "n12")
    evk_t = dev(g, evk)
    for level in (3, 2, 1):
        c1 = np.ascontiguousarray(np.stack([ct1[0, :level], ct1[1, :level]]))
        c2 = np.ascontiguousarray(np.stack([ct2[0, :level], ct2[1, :level]]))
        want = oracle.he_mul(op, c1, c2, evk, level)
        assert np.array_equal(gpu_mul(g, ctx, c1, c2, evk_t, level, fused=False), want), level
        if level >= 2:
            want_rs = oracle.rescale(op, want, level)
            assert np.array_equal(gpu_mul(g, ctx, c1, c2, evk_t, level, fused=True), want_rs), level
            out = torch.empty((2, level - 1, op.N), dtype=torch.int64, device="cuda")
            g.he_rescale(ctx, dev(g, want), level, out, g.workspace(ctx, level))
            torch.cuda.synchronize()
            assert np.array_equal(host(g, out), want_rs), level
    # and the GPU result decrypts to m1*m2
    res = gpu_mul(g, ctx, ct1, ct2, evk_t, op.L, fused=True)
    z = oracle.decrypt(op, sk, res, op.L - 1, sc * sc / int(op.q[op.L - 1]))
    assert np.abs(z - m1 * m2).max() < 2.0 ** -14


def test_he_mul_n16_full_level_real_keys(g):
    op, sc, sk, pk, evk, m1, m2, ct1, ct2 = real_inputs("n16")
    ctx = ctx_for(g, "n16")
    evk_t = dev(g, evk)
    want = oracle.he_mul(op, ct1, ct2, evk, op.L)
    assert np.array_equal(gpu_mul(g, ctx, ct1, ct2, evk_t, op.L, fused=False), want)
    want_rs = oracle.rescale(op, want, op.L)
    got = gpu_mul(g, ctx, ct1, ct2, evk_t, op.L, fused=True)
    assert np.array_equal(got, want_rs)
    z = oracle.decrypt(op, sk, got, op.L - 1, sc * sc / int(op.q[op.L - 1]))
    err = np.abs(z - m1 * m2).max()
    assert 2.0 ** -60 < err < 2.0 ** -24


@pytest.mark.parametrize("name,level", [("n16", 13), ("n16", 2), ("n15", 16), ("n15", 9)])
def test_he_mul_rescale_ragged_levels(g, name, level):
    ctx = ctx_for(g, name)
    op = oracle.preset(name)
    ct1, ct2 = rand_ct(op, level, 71), rand_ct(op, level, 73)
    evk = rand_evk(op, 80)
    want = oracle.rescale(op, oracle.he_mul(op, ct1, ct2, evk, level), level)
    assert np.array_equal(gpu_mul(g, ctx, ct1, ct2, dev(g, evk), level, fused=True), want)


@pytest.mark.slow
def test_he_mul_rescale_n17_full(g):
    ctx = ctx_for(g, "n17")
    op = oracle.preset("n17")
    level = op.L
    ct1, ct2 = rand_ct(op, level, 91), rand_ct(op, level, 93)
    evk = rand_evk(op, 100)
    want = oracle.rescale(op, oracle.he_mul(op, ct1, ct2, evk, level), level)
    evk_t = dev(g, evk)
    assert np.array_equal(gpu_mul(g, ctx, ct1, ct2, evk_t, level, fused=True), want)
    try:  # four digits: the special rows' sums inside their iNTT's first pass
        g.he_set_shape(ctx, 1, 16, 1, 9, 8, 7, 1)
        assert np.array_equal(gpu_mul(g, ctx, ct1, ct2, evk_t, level, fused=True), want)
    finally:
        g.he_set_shape(ctx, 4, 8, 1)


def test_batch_matches_single_and_oracle(g):
    import torch
    name = "n16"
    ctx = ctx_for(g, name)
    op = oracle.preset(name)
    evk = rand_evk(op, 120)
    evk_t = dev(g, evk)
    levels = [4, 24, 9, 17, 2, 13]
    jobs, singles, cts = [], [], []
    for k, lv in enumerate(levels):
        c1, c2 = rand_ct(op, lv, 200 + 2 * k), rand_ct(op, lv, 300 + 2 * k)
        cts.append((c1, c2))
        t1, t2 = dev(g, c1), dev(g, c2)
        out = torch.empty((2, lv - 1, op.N), dtype=torch.int64, device="cuda")
        jobs.append((t1, t2, out, lv))
        singles.append(gpu_mul(g, ctx, c1, c2, evk_t, lv, fused=True))
    nbytes = g.he_batch_workspace_bytes(ctx, levels)
    ws = torch.empty(nbytes // 8, dtype=torch.int64, device="cuda")
    g.he_mul_batch(ctx, jobs, evk_t, ws)
    torch.cuda.synchronize()
    for (t1, t2, out, lv), single in zip(jobs, singles):
        assert np.array_equal(host(g, out), single), lv
    for k in (0, 4):  # two entries against the oracle directly
        c1, c2 = cts[k]
        lv = levels[k]
        want = oracle.rescale(op, oracle.he_mul(op, c1, c2, evk, lv), lv)
        assert np.array_equal(host(g, jobs[k][2]), want)


@pytest.mark.parametrize("levels,ip_jobs,fuse,pdl", [
    ([3, 5], 8, 1, 1), ([5, 3], 4, 0, 2), ([3, 5, 2, 4, 5, 3, 2, 8, 9], 4, 1, 2),
    ([24, 4, 9, 17, 2, 13, 24, 23, 16, 8, 3], 8, 1, 2), ([24, 9, 17, 2], 1, 0, 0), ([24, 9, 17, 2], 1, 1, 1)])
def test_batch_shared_key_words_bit_exact(g, levels, ip_jobs, fuse, pdl):
    """Batches whose inner product shares each CTA's evaluation-key words among
    up to ip_jobs jobs of similar level (groups cut from the jobs sorted by
    level, ragged last group, jobs of a group at different levels and digit
    counts): every result equals he_mul_rescale on the job alone, bit for bit,
    and the lowest-level job equals the oracle."""
    import torch
    name = "n16"
    ctx = ctx_for(g, name)
    op = oracle.preset(name)
    evk = rand_evk(op, 160)
    evk_t = dev(g, evk)
    jobs, singles, cts = [], [], []
    for k, lv in enumerate(levels):
        c1, c2 = rand_ct(op, lv, 1200 + 2 * k), rand_ct(op, lv, 1300 + 2 * k)
        cts.append((c1, c2))
        out = torch.full((2, lv - 1, op.N), -1, dtype=torch.int64, device="cuda")
        jobs.append((dev(g, c1), dev(g, c2), out, lv))
        singles.append(gpu_mul(g, ctx, c1, c2, evk_t, lv, fused=True))
    ws = torch.empty(g.he_batch_workspace_bytes(ctx, levels) // 8, dtype=torch.int64, device="cuda")
    try:
        g.he_set_shape(ctx, 4, 8, pdl, 0, ip_jobs, fuse)
        for rnd in range(2):  # twice on the same workspace
            for j in jobs:
                j[2].fill_(-1)
            g.he_mul_batch(ctx, jobs, evk_t, ws)
            torch.cuda.synchronize()
            for (t1, t2, out, lv), single in zip(jobs, singles):
                assert np.array_equal(host(g, out), single), (rnd, lv)
    finally:
        g.he_set_shape(ctx, 4, 8, 1)
    k = int(np.argmin(levels))
    c1, c2 = cts[k]
    want = oracle.rescale(op, oracle.he_mul(op, c1, c2, evk, levels[k]), levels[k])
    assert np.array_equal(host(g, jobs[k][2]), want)


@pytest.mark.parametrize("capture_cap,replay_cap,pdl", [(4, 4, 1), (1, 3, 2), (4, 1, 2)])
def test_batch_graph_replays_match_single(g, capture_cap, replay_cap, pdl):
    """One captured graph, replayed with two different batches (sizes, levels,
    operands): every result equals he_mul_rescale on the job alone.  Captured
    at limb-group cap 1 (single-buffered NTT tiles) and replayed at cap 3, the
    NTT kernels get groups of several limbs and load them one after another."""
    import torch
    name = "n16"
    ctx = ctx_for(g, name)
    op = oracle.preset(name)
    evk_t = dev(g, rand_evk(op, 130))
    g.he_set_shape(ctx, capture_cap, 8, pdl)
    graph = g.BatchGraph(ctx, 8, evk_t)
    g.he_set_shape(ctx, replay_cap, 8, pdl)
    for rnd, levels in enumerate([[24, 5, 13, 2, 18, 9], [3, 24, 11]]):
        jobs, singles = [], []
        for k, lv in enumerate(levels):
            c1, c2 = rand_ct(op, lv, 400 + 10 * rnd + 2 * k), rand_ct(op, lv, 500 + 10 * rnd + 2 * k)
            out = torch.full((2, lv - 1, op.N), -1, dtype=torch.int64, device="cuda")
            jobs.append((dev(g, c1), dev(g, c2), out, lv))
            singles.append(gpu_mul(g, ctx, c1, c2, evk_t, lv, fused=True))
        graph.launch(jobs)
        torch.cuda.synchronize()
        for (t1, t2, out, lv), single in zip(jobs, singles):
            assert np.array_equal(host(g, out), single), (rnd, lv)
    with pytest.raises(g.HeError):
        graph.launch([jobs[0]] * 9)  # more jobs than captured
    graph.close()
    g.he_set_shape(ctx, 4, 8, 1)


def test_server_continuous_batching_matches_single(g):
    """Requests of two rings and many levels, submitted while earlier ones run,
    under an HBM budget that admits only a few at a time: every result is the
    same as the request run alone."""
    import torch
    rings = ["n15", "n16"]
    ctxs = [ctx_for(g, r) for r in rings]
    ops = [oracle.preset(r) for r in rings]
    evks = [dev(g, rand_evk(op, 140 + i)) for i, op in enumerate(ops)]
    # room for roughly four level-16 N=2^16 requests at once
    budget = 4 * g.he_batch_workspace_bytes(ctxs[1], [16])
    srv = g.Server(ctxs, evks, hbm_budget=budget, max_batch=8, streams=3)
    rng = np.random.default_rng(9)
    staged = []
    for k in range(40):
        ri = int(rng.random() < 0.3)
        op = ops[ri]
        lv = int(rng.integers(2, 17)) if ri == 0 else int(rng.integers(4, 25))
        c1, c2 = rand_ct(op, lv, 600 + 2 * k), rand_ct(op, lv, 700 + 2 * k)
        out = torch.full((2, lv - 1, op.N), -1, dtype=torch.int64, device="cuda")
        staged.append((ri, lv, dev(g, c1), dev(g, c2), out))
    torch.cuda.synchronize()
    # submit back to back: later requests arrive while earlier batches run
    reqs = [(ri, lv, t1, t2, out, srv.submit(ri, lv, t1, t2, out)) for ri, lv, t1, t2, out in staged]
    for ri, lv, t1, t2, out, tk in reqs:
        srv.wait(tk, 120000)
        assert srv.poll(tk)
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["pending"] == 0
    assert st["batches"] < len(reqs)  # requests were batched
    assert 0 < st["p50_ms"] <= st["p99_ms"]
    srv.close()
    for ri, lv, t1, t2, out, tk in reqs:
        ctx = ctxs[ri]
        alone = torch.empty_like(out)
        g.he_mul_rescale(ctx, t1, t2, evks[ri], lv, alone, g.workspace(ctx, lv))
        torch.cuda.synchronize()
        assert torch.equal(out, alone), (ri, lv)


def test_server_admission_errors(g):
    import torch
    ctx = ctx_for(g, "n16")
    op = oracle.preset("n16")
    evk = dev(g, rand_evk(op, 150))
    small = g.he_batch_workspace_bytes(ctx, [8])
    srv = g.Server([ctx], [evk], hbm_budget=small, max_batch=4, streams=2)
    a = torch.zeros((2, 24, op.N), dtype=torch.int64, device="cuda")
    out = torch.zeros((2, 23, op.N), dtype=torch.int64, device="cuda")
    with pytest.raises(g.HeError) as e:  # a level-24 request never fits this budget
        srv.submit(0, 24, a, a, out)
    assert e.value.code == g.HE_ENOMEM
    with pytest.raises(g.HeError) as e:
        srv.submit(0, 1, a, a, out)
    assert e.value.code == g.HE_ELEVEL
    b = torch.zeros((2, 8, op.N), dtype=torch.int64, device="cuda")
    o2 = torch.zeros((2, 7, op.N), dtype=torch.int64, device="cuda")
    # the budget admits one level-8 request at a time: the last of eight
    # queued back to back waits behind seven HE Muls run one after another,
    # so a zero-timeout wait on it right after submitting must time out
    tks = [srv.submit(0, 8, b, b, o2) for _ in range(8)]
    assert g.lib().he_server_wait(srv.ptr, tks[-1], 0) == g.HE_ETIMEOUT
    for tk in tks:
        srv.wait(tk, 60000)
    assert g.lib().he_server_wait(srv.ptr, tks[-1], 0) == g.HE_OK
    st = srv.stats()
    assert st["batches"] == 8 and st["completed"] == 8  # one request per batch under this budget
    with pytest.raises(g.HeError) as e:
        srv.poll(123456789)  # never issued
    assert e.value.code == g.HE_EINVAL
    srv.close()


def test_server_waits_for_request_events(g):
    """Operands written on another stream and submitted at once, with the
    event recorded after the writes: the batch waits for the event on the
    device, and the result equals he_mul_rescale on the same operands."""
    import torch
    ctx = ctx_for(g, "n16")
    op = oracle.preset("n16")
    evk_t = dev(g, rand_evk(op, 170))
    lv = 20
    srv = g.Server([ctx], [evk_t], hbm_budget=2 * g.he_batch_workspace_bytes(ctx, [lv]), max_batch=4, streams=2)
    src1, src2 = dev(g, rand_ct(op, lv, 1400)), dev(g, rand_ct(op, lv, 1402))
    writer = torch.cuda.Stream()
    torch.cuda.synchronize()
    a, b = torch.empty_like(src1), torch.empty_like(src2)
    out = torch.full((2, lv - 1, op.N), -1, dtype=torch.int64, device="cuda")
    with torch.cuda.stream(writer):
        for _ in range(20):  # keep the writer busy for a while before the copies land
            a.copy_(src2)
            b.copy_(src1)
        a.copy_(src1)
        b.copy_(src2)
        ev = torch.cuda.Event()
        ev.record(writer)
    tk = srv.submit(0, lv, a, b, out, ready=ev)
    srv.wait(tk, 60000)
    torch.cuda.synchronize()
    ref = torch.empty_like(out)
    g.he_mul_rescale(ctx, src1, src2, evk_t, lv, ref, g.workspace(ctx, lv))
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    srv.close()


def test_device_argument_errors(g):
    import torch
    ctx = ctx_for(g, "n12")
    N = ctx.N
    a = torch.zeros((2, 3, N), dtype=torch.int64, device="cuda")
    out = torch.zeros((2, 3, N), dtype=torch.int64, device="cuda")
    ws = g.workspace(ctx, 3)
    small = ws[: ws.numel() // 2]
    with pytest.raises(g.HeError) as e:
        g.he_mul(ctx, a, a, a, 3, out, small)
    assert e.value.code == g.HE_ENOMEM
    with pytest.raises(g.HeError) as e:
        g.he_mul(ctx, a, a, a, 4, out, ws)
    assert e.value.code == g.HE_ELEVEL
    with pytest.raises(g.HeError) as e:
        g.he_rescale(ctx, a, 1, out, ws)
    assert e.value.code == g.HE_ELEVEL
    mis = torch.zeros(2 * 3 * N + 1, dtype=torch.int64, device="cuda")[1:]
    rc = g.lib().he_mul(ctx.ptr, mis.data_ptr(), a.data_ptr(), a.data_ptr(), 3, out.data_ptr(), ws.data_ptr(),
                        ws.numel() * 8, None)
    assert rc == g.HE_EINVAL


# ---------------------------------------------------------------------------
# rotation (Galois automorphism + key switching with a rotation key)
# ---------------------------------------------------------------------------
def gpu_rotate(g, ctx, ct, rk_t, level, gal):
    import torch
    out = torch.empty((2, level, ctx.N), dtype=torch.int64, device="cuda")
    g.he_rotate(ctx, dev(g, ct), rk_t, level, gal, out, g.workspace(ctx, level))
    torch.cuda.synchronize()
    return host(g, out)


def test_rotate_n12_every_level_and_conjugate(g):
    op, sc, sk, pk, evk, m1, m2, ct1, ct2 = real_inputs("n12")
    ctx = ctx_for(g, "n12")
    for steps in (1, -1, 5):
        gal = oracle.galois_elt(op, steps)
        rk = oracle.keygen_rot(op, sk, gal, 900 + steps % 50)
        rk_t = dev(g, rk)
        for level in (3, 2, 1):
            c = np.ascontiguousarray(np.stack([ct1[0, :level], ct1[1, :level]]))
            assert np.array_equal(gpu_rotate(g, ctx, c, rk_t, level, gal), oracle.rotate(op, c, gal, rk, level)), \
                (steps, level)
        z = oracle.decrypt(op, sk, gpu_rotate(g, ctx, ct1, rk_t, op.L, gal), op.L, sc)
        assert np.abs(z - np.roll(m1, -steps)).max() < 2.0 ** -16
    gal = oracle.conj_elt(op)
    rk = oracle.keygen_rot(op, sk, gal, 950)
    got = gpu_rotate(g, ctx, ct2, dev(g, rk), op.L, gal)
    assert np.array_equal(got, oracle.rotate(op, ct2, gal, rk, op.L))
    assert np.abs(oracle.decrypt(op, sk, got, op.L, sc) - np.conj(m2)).max() < 2.0 ** -16


@pytest.mark.parametrize("level", [24, 13])
def test_rotate_n16_real_keys(g, level):
    op, sc, sk, pk, evk, m1, m2, ct1, ct2 = real_inputs("n16")
    ctx = ctx_for(g, "n16")
    gal = oracle.galois_elt(op, 3)
    rk = oracle.keygen_rot(op, sk, gal, 1611)
    c = np.ascontiguousarray(np.stack([ct1[0, :level], ct1[1, :level]]))
    got = gpu_rotate(g, ctx, c, dev(g, rk), level, gal)
    assert np.array_equal(got, oracle.rotate(op, c, gal, rk, level))
    z = oracle.decrypt(op, sk, got, level, sc)
    assert np.abs(z - np.roll(m1, -3)).max() < 2.0 ** -24


def test_rotate_argument_errors(g):
    import torch
    ctx = ctx_for(g, "n12")
    N = ctx.N
    a = torch.zeros((2, 3, N), dtype=torch.int64, device="cuda")
    out = torch.zeros((2, 3, N), dtype=torch.int64, device="cuda")
    rk = torch.zeros((ctx.dnum, 2, ctx.prm.K + ctx.prm.L, N), dtype=torch.int64, device="cuda")
    ws = g.workspace(ctx, 3)
    for bad_g, code in ((2, g.HE_EINVAL), (2 * N + 1, g.HE_EINVAL)):
        with pytest.raises(g.HeError) as e:
            g.he_rotate(ctx, a, rk, 3, bad_g, out, ws)
        assert e.value.code == code
    with pytest.raises(g.HeError) as e:
        g.he_rotate(ctx, a, rk, 4, 5, out, ws)
    assert e.value.code == g.HE_ELEVEL
    with pytest.raises(g.HeError) as e:
        g.he_rotate(ctx, a, rk, 3, 5, out, ws[: ws.numel() // 2])
    assert e.value.code == g.HE_ENOMEM


# ---------------------------------------------------------------------------
# HE Add / Sub, plaintext ops, and a multiplication chain down the levels
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name,level", [("n12", 3), ("n16", 24), ("n16", 7)])
def test_add_sub_plain_ops(g, name, level):
    import torch
    ctx = ctx_for(g, name)
    op = oracle.preset(name)
    c1, c2 = rand_ct(op, level, 301), rand_ct(op, level, 303)
    c1[:, :, :3] = np.array([int(q) - 1 for q in op.q[:level]], dtype=np.uint64)[None, :, None]
    c2[:, :, :3] = np.array([int(q) - 1 for q in op.q[:level]], dtype=np.uint64)[None, :, None]
    rng = np.random.default_rng(level)
    t = rng.integers(-(1 << 60), 1 << 60, size=op.N, dtype=np.int64)
    pt = oracle.plain_ntt(op, t, level)
    a, b, p = dev(g, c1), dev(g, c2), dev(g, pt)
    out = torch.empty_like(a)
    cases = [(g.he_add, b, oracle.add(op, c1, c2, level)), (g.he_sub, b, oracle.sub(op, c1, c2, level)),
             (g.he_mul_plain, p, oracle.mul_plain(op, c1, pt, level)),
             (g.he_add_plain, p, oracle.add_plain(op, c1, pt, level))]
    for fn, y, want in cases:
        fn(ctx, a, y, level, out)
        torch.cuda.synchronize()
        assert np.array_equal(host(g, out), want), fn.__name__
    # in place (out aliases the first operand)
    a2 = a.clone()
    g.he_add(ctx, a2, b, level, a2)
    torch.cuda.synchronize()
    assert np.array_equal(host(g, a2), oracle.add(op, c1, c2, level))


def test_squaring_chain_n12_decrypts(g):
    """Scale q_{L-1}; HE Mul + rescale at every level down to level 1, bit-exact
    to the oracle at each level and decrypting to m^(2^k)."""
    import torch
    op, sc, sk, pk, evk, m1, m2, ct1, ct2 = real_inputs("n12")
    ctx = ctx_for(g, "n12")
    evk_t = dev(g, evk)
    m = 0.5 * m1
    L = op.L
    scale = float(int(op.q[L - 1]))
    ct = oracle.encrypt_poly(op, pk, encode(m, op.logN, scale), L, 1211)
    cur = dev(g, ct)
    want_ct, want = ct, m
    for l in range(L, 1, -1):
        nxt = torch.empty((2, l - 1, op.N), dtype=torch.int64, device="cuda")
        g.he_mul_rescale(ctx, cur, cur, evk_t, l, nxt, g.workspace(ctx, l))
        torch.cuda.synchronize()
        want_ct = oracle.rescale(op, oracle.he_mul(op, want_ct, want_ct, evk, l), l)
        got = host(g, nxt)
        assert np.array_equal(got, want_ct), l
        scale = scale * scale / int(op.q[l - 1])
        want = want * want
        assert np.abs(oracle.decrypt(op, sk, got, l - 1, scale) - want).max() < 2.0 ** -12
        cur = nxt


@pytest.mark.slow
def test_squaring_chain_n15_all_levels(g):
    """N=2^15, 16 levels: 15 HE Mul + rescale steps, bit-exact at every level."""
    import torch
    name = "n15"
    ctx = ctx_for(g, name)
    op = oracle.preset(name)
    ks = si.SEEDS[name][0]
    sk = oracle.keygen_sk(op, ks)
    pk = oracle.keygen_pk(op, sk, ks)
    evk = oracle.keygen_evk(op, sk, ks)
    m = 0.5 * si.messages(op.N // 2, 1512)
    L = op.L
    scale = float(int(op.q[L - 1]))
    want_ct = oracle.encrypt_poly(op, pk, encode(m, op.logN, scale), L, 1513)
    cur, evk_t = dev(g, want_ct), dev(g, evk)
    want = m
    for l in range(L, 1, -1):
        nxt = torch.empty((2, l - 1, op.N), dtype=torch.int64, device="cuda")
        g.he_mul_rescale(ctx, cur, cur, evk_t, l, nxt, g.workspace(ctx, l))
        torch.cuda.synchronize()
        want_ct = oracle.rescale(op, oracle.he_mul(op, want_ct, want_ct, evk, l), l)
        assert np.array_equal(host(g, nxt), want_ct), l
        scale = scale * scale / int(op.q[l - 1])
        want = want * want
        cur = nxt
    z = oracle.decrypt(op, sk, host(g, cur), 1, scale)
    assert np.abs(z - want).max() < 2.0 ** -20



# ---------------------------------------------------------------------------
# launch shapes and the autotuner: speed only, bits unchanged
# ---------------------------------------------------------------------------
def test_every_shape_is_bit_identical_n16(g):
    op, sc, sk, pk, evk, m1, m2, ct1, ct2 = real_inputs("n16")
    ctx = ctx_for(g, "n16")
    evk_t = dev(g, evk)
    level = 17
    c1 = np.ascontiguousarray(np.stack([ct1[0, :level], ct1[1, :level]]))
    c2 = np.ascontiguousarray(np.stack([ct2[0, :level], ct2[1, :level]]))
    want = oracle.rescale(op, oracle.he_mul(op, c1, c2, evk, level), level)
    try:
        for shape in ((1, 4, 1, 15), (2, 16, 0, 5), (3, 8, 1, 10), (4, 16, 0, 0), (4, 8, 1, 0), (1, 8, 1, 3),
                      (1, 8, 1, 8, 8, 0), (3, 4, 0, 1, 8, 0), (2, 8, 1, 15, 8, 0), (1, 8, 2, 9, 8, 1),
                      (4, 16, 2, 0, 8, 0), (1, 8, 2, 9, 8, 2), (2, 16, 1, 6, 8, 3), (1, 4, 0, 0, 8, 2),
                      (1, 8, 2, 15, 8, 7, 1, 1), (3, 8, 1, 0, 8, 6), (2, 16, 0, 5, 8, 7, 2), (1, 8, 1, 15, 8, 5)):
            g.he_set_shape(ctx, *shape)
            assert np.array_equal(gpu_mul(g, ctx, c1, c2, evk_t, level, fused=True), want), shape
        want_plain = oracle.he_mul(op, c1, c2, evk, level)
        for fz in (1, 0):  # the plain ModDown path with the radix-8 plans, tensor fused or not
            g.he_set_shape(ctx, 2, 8, 1, 15, 8, fz)
            assert np.array_equal(gpu_mul(g, ctx, c1, c2, evk_t, level, fused=False), want_plain), fz
    finally:
        g.he_set_shape(ctx, 4, 8, 1)


@pytest.mark.parametrize("name,level,split", [("n16", 24, 0), ("n16", 24, 1), ("n16", 9, 2), ("n17", 44, 1),
                                              ("n17", 13, 2)])
def test_ntt_pass_splits_bit_identical(g, name, level, split):
    """Every NTT of the path on a pass split (one stage moved between the
    strided and the contiguous pass), in the radix-16 and the radix-8 form,
    on 2048- and 1024-element tiles (all sites, or sites 1 and 3): the same
    words as the oracle.  The raw transforms too (he_step_ntt takes the
    context's split and site 0's radix and tile bits)."""
    import torch
    op = oracle.preset(name)
    ctx = ctx_for(g, name)
    evk = rand_evk(op, 930 + level)
    evk_t = dev(g, evk)
    c1, c2 = rand_ct(op, level, 940 + level), rand_ct(op, level, 950 + level)
    want = oracle.rescale(op, oracle.he_mul(op, c1, c2, evk, level), level)
    try:
        for r8 in (0, 15, 5):
            for small in (0, 15, 10):
                fz = 7 if small == 10 else 3  # and the special rows' sums inside their iNTT
                g.he_set_shape(ctx, 1, 8, 1, r8, 8, fz, split, small)
                assert np.array_equal(gpu_mul(g, ctx, c1, c2, evk_t, level, fused=True), want), (split, r8, small)
        E = op.K + op.L
        idx = [0, op.K, E - 1]
        mods = [op.ext[e] for e in idx]
        psis = [int(op.psi_p[e]) if e < op.K else int(op.psi_q[e - op.K]) for e in idx]
        a = rand_polys(mods, op.N, 960 + split)
        for r8, small in ((0, 0), (1, 0), (0, 1), (1, 1)):
            g.he_set_shape(ctx, 1, 8, 1, r8, 8, 3, split, small)
            t = dev(g, a)
            g.he_step_ntt(ctx, t, idx, inverse=False)
            torch.cuda.synchronize()
            assert np.array_equal(host(g, t), np.stack([oracle.ntt(a[i], mods[i], psis[i], op.logN)
                                                        for i in range(len(idx))])), (split, r8, small)
            g.he_step_ntt(ctx, t, idx, inverse=True)
            torch.cuda.synchronize()
            assert np.array_equal(host(g, t), a), (split, r8, small)
    finally:
        g.he_set_shape(ctx, 4, 8, 1)


@pytest.mark.parametrize("name,levels", [("n16", (2, 3, 8, 9)), ("n15", (2, 5)), ("n12", (2, 3))])
def test_fused_special_sums_low_levels(g, name, levels):
    """The special rows' key-switch sums inside their iNTT's first pass (fuse
    bit 2) at the lowest levels and at digit boundaries (a short last digit,
    q_{l-1} in the first digit), on every ring size's plans: the oracle's words."""
    op = oracle.preset(name)
    ctx = ctx_for(g, name)
    evk = rand_evk(op, 1010)
    evk_t = dev(g, evk)
    try:
        for level in levels:
            c1, c2 = rand_ct(op, level, 1020 + level), rand_ct(op, level, 1040 + level)
            want = oracle.rescale(op, oracle.he_mul(op, c1, c2, evk, level), level)
            for shape in ((1, 8, 2, 15, 8, 7), (3, 4, 1, 0, 8, 7)):
                g.he_set_shape(ctx, *shape)
                assert np.array_equal(gpu_mul(g, ctx, c1, c2, evk_t, level, fused=True), want), (level, shape)
    finally:
        g.he_set_shape(ctx, 4, 8, 1)


@pytest.mark.parametrize("level", [24, 3])
def test_onepass_cluster_bit_identical(g, level):
    """The one-pass transforms over a cluster of 8 CTAs (N = 2^16) at every
    NTT site or at some, the other sites on radix-8 or radix-16 passes, with
    and without the fusions (the tensor product in the first iNTT, the final
    combine in the last NTT) and with groups of 1 to 4 limbs per cluster: the
    same words as the oracle; the plain ModDown path and the raw transforms
    (he_step_ntt takes site 0's bit) too."""
    import torch
    name = "n16"
    op = oracle.preset(name)
    ctx = ctx_for(g, name)
    evk = rand_evk(op, 970 + level)
    evk_t = dev(g, evk)
    c1, c2 = rand_ct(op, level, 980 + level), rand_ct(op, level, 990 + level)
    want = oracle.rescale(op, oracle.he_mul(op, c1, c2, evk, level), level)
    try:
        for onepass in (15, 5, 10):
            for r8, fz, grp in ((15, 3, 1), (0, 0, 2), (5, 1, 4)):
                g.he_set_shape(ctx, grp, 8, 1, r8, 8, fz, 1, 0, onepass)
                got = gpu_mul(g, ctx, c1, c2, evk_t, level, fused=True)
                assert np.array_equal(got, want), (onepass, r8, fz, grp)
        g.he_set_shape(ctx, 2, 8, 2, 15, 8, 1, 0, 0, 15)
        assert np.array_equal(gpu_mul(g, ctx, c1, c2, evk_t, level, fused=False), oracle.he_mul(op, c1, c2, evk, level))
        E = op.K + op.L
        idx = [0, op.K, E - 1]
        mods = [op.ext[e] for e in idx]
        psis = [int(op.psi_p[e]) if e < op.K else int(op.psi_q[e - op.K]) for e in idx]
        a = rand_polys(mods, op.N, 975 + level)
        for grp in (1, 3):
            g.he_set_shape(ctx, grp, 8, 1, 0, 8, 3, 0, 0, 1)
            t = dev(g, a)
            g.he_step_ntt(ctx, t, idx, inverse=False)
            torch.cuda.synchronize()
            assert np.array_equal(host(g, t), np.stack([oracle.ntt(a[i], mods[i], psis[i], op.logN)
                                                        for i in range(len(idx))])), grp
            g.he_step_ntt(ctx, t, idx, inverse=True)
            torch.cuda.synchronize()
            assert np.array_equal(host(g, t), a), grp
    finally:
        g.he_set_shape(ctx, 4, 8, 1)


def test_onepass_batch_and_graph_match_single(g):
    """A batch of uneven levels and a graph replay (NTT grids resized to each
    batch) on one-pass shapes: every result equals the job run alone."""
    import torch
    name = "n16"
    ctx = ctx_for(g, name)
    op = oracle.preset(name)
    evk_t = dev(g, rand_evk(op, 125))
    levels = [24, 5, 13, 2, 18]
    try:
        g.he_set_shape(ctx, 2, 8, 2, 15, 8, 3, 1, 0, 15)
        graph = g.BatchGraph(ctx, 8, evk_t)
        jobs, singles = [], []
        for k, lv in enumerate(levels):
            c1, c2 = rand_ct(op, lv, 600 + 2 * k), rand_ct(op, lv, 650 + 2 * k)
            jobs.append((dev(g, c1), dev(g, c2), torch.full((2, lv - 1, op.N), -1, dtype=torch.int64, device="cuda"), lv))
            singles.append(gpu_mul(g, ctx, c1, c2, evk_t, lv, fused=True))
        ws = torch.empty(g.he_batch_workspace_bytes(ctx, levels) // 8, dtype=torch.int64, device="cuda")
        g.he_mul_batch(ctx, jobs, evk_t, ws)
        torch.cuda.synchronize()
        for (t1, t2, out, lv), single in zip(jobs, singles):
            assert np.array_equal(host(g, out), single), lv
            out.fill_(-1)
        graph.launch(jobs[:3])
        torch.cuda.synchronize()
        for (t1, t2, out, lv), single in zip(jobs[:3], singles[:3]):
            assert np.array_equal(host(g, out), single), lv
        graph.close()
    finally:
        g.he_set_shape(ctx, 4, 8, 1)


@pytest.mark.parametrize("name,level", [("n15", 16), ("n15", 5), ("n17", 13)])
def test_radix8_plans_bit_identical(g, name, level):
    """Every NTT site on its radix-8 plan (the plans differ per ring size)."""
    op = oracle.preset(name)
    ctx = ctx_for(g, name)
    evk = rand_evk(op, 900 + level)
    evk_t = dev(g, evk)
    c1, c2 = rand_ct(op, level, 910 + level), rand_ct(op, level, 920 + level)
    try:
        g.he_set_shape(ctx, 1, 8, 1, 15)
        want = oracle.rescale(op, oracle.he_mul(op, c1, c2, evk, level), level)
        assert np.array_equal(gpu_mul(g, ctx, c1, c2, evk_t, level, fused=True), want)
    finally:
        g.he_set_shape(ctx, 4, 8, 1)


def test_autotune_batch_keeps_results(g):
    import torch
    ctx = ctx_for(g, "n15")
    op = oracle.preset("n15")
    evk = rand_evk(op, 700)
    evk_t = dev(g, evk)
    levels = [16, 9, 3, 12]
    jobs, want = [], []
    for k, lv in enumerate(levels):
        a, b = rand_ct(op, lv, 710 + 4 * k), rand_ct(op, lv, 712 + 4 * k)
        jobs.append((dev(g, a), dev(g, b), torch.empty((2, lv - 1, op.N), dtype=torch.int64, device="cuda"), lv))
        want.append(oracle.rescale(op, oracle.he_mul(op, a, b, evk, lv), lv))
    ws = torch.empty(g.he_batch_workspace_bytes(ctx, levels) // 8, dtype=torch.int64, device="cuda")
    try:
        best, tried = g.he_autotune(ctx, jobs, evk_t, ws, reps=2)
        assert all(t[9] > 0 for t in tried) and len(set(t[:9] for t in tried)) == len(tried)
        # the kept shape is one of the four fastest of the search, re-timed
        fastest = sorted(tried, key=lambda t: t[9])[:4]
        assert best[:9] == g.he_get_shape(ctx) and best[:9] in {t[:9] for t in fastest} and best[9] > 0
        # the first sweep gives every knob every value (N = 2^15: no pass splits
        # or small tiles); pdl with fuse and ntt_r8 with ntt_split take every pair
        for k, vals in enumerate(((1, 2, 3, 4), (4, 8, 16), (0, 1, 2), tuple(range(16)), (1, 4, 8), (0, 1, 2, 3), (0,),
                                  (0,), (0,))):
            assert set(vals) <= {t[k] for t in tried}, k
        assert {(p, f) for p in range(3) for f in range(4)} <= {(t[2], t[5]) for t in tried}
        for j in jobs:
            j[2].zero_()
        g.he_mul_batch(ctx, jobs, evk_t, ws)
        torch.cuda.synchronize()
        for j, w in zip(jobs, want):
            assert np.array_equal(host(g, j[2]), w)
        g.he_set_shape(ctx, 2, 8, 1, 15)  # the batch on the radix-8 plans
        for j in jobs:
            j[2].zero_()
        g.he_mul_batch(ctx, jobs, evk_t, ws)
        torch.cuda.synchronize()
        for j, w in zip(jobs, want):
            assert np.array_equal(host(g, j[2]), w)
    finally:
        g.he_set_shape(ctx, 4, 8, 1)



# ---------------------------------------------------------------------------
# seeded evaluation key: b halves on the device, a halves regenerated
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name,levels", [("n12", (3, 2)), ("n16", (24, 9))])
def test_seeded_key_he_mul_bit_exact(g, name, levels):
    import torch
    op, sc, sk, pk, evk, m1, m2, ct1, ct2 = real_inputs(name)
    ctx = ctx_for(g, name)
    seed = 5150
    full = oracle.keygen_evk_seeded(op, sk, seed)
    evk_b = dev(g, np.ascontiguousarray(full[:, 0]))
    g.he_evk_register_seeded(ctx, evk_b, seed)
    try:
        for level in levels:
            c1 = np.ascontiguousarray(np.stack([ct1[0, :level], ct1[1, :level]]))
            c2 = np.ascontiguousarray(np.stack([ct2[0, :level], ct2[1, :level]]))
            want = oracle.he_mul(op, c1, c2, full, level)
            assert np.array_equal(gpu_mul(g, ctx, c1, c2, evk_b, level, fused=False), want), level
            got = gpu_mul(g, ctx, c1, c2, evk_b, level, fused=True)
            assert np.array_equal(got, oracle.rescale(op, want, level)), level
            g.he_set_shape(ctx, 4, 8, 1, 0, 8, 7)  # a seeded key keeps its own sums kernel
            assert np.array_equal(gpu_mul(g, ctx, c1, c2, evk_b, level, fused=True), got), level
            g.he_set_shape(ctx, 4, 8, 1)
        z = oracle.decrypt(op, sk, got, levels[-1] - 1, sc * sc / int(op.q[levels[-1] - 1]))
        assert np.abs(z - m1 * m2).max() < (2.0 ** -14 if name == "n12" else 2.0 ** -24)
        # the same jobs batched
        jobs, want = [], []
        for level in levels:
            c1 = np.ascontiguousarray(np.stack([ct1[0, :level], ct1[1, :level]]))
            c2 = np.ascontiguousarray(np.stack([ct2[0, :level], ct2[1, :level]]))
            jobs.append((dev(g, c1), dev(g, c2), torch.empty((2, level - 1, op.N), dtype=torch.int64, device="cuda"),
                         level))
            want.append(oracle.rescale(op, oracle.he_mul(op, c1, c2, full, level), level))
        ws = torch.empty(g.he_batch_workspace_bytes(ctx, list(levels)) // 8, dtype=torch.int64, device="cuda")
        g.he_mul_batch(ctx, jobs, evk_b, ws)
        torch.cuda.synchronize()
        for j, w in zip(jobs, want):
            assert np.array_equal(host(g, j[2]), w)
    finally:
        g.he_evk_unregister(ctx, evk_b)


# ---------------------------------------------------------------------------
# measurement probes (the ALU ceilings the bench grades kernels against)
# ---------------------------------------------------------------------------
def test_probes_run_and_reject_bad_arguments(g):
    bfly = g.he_probe_butterfly_rate(152, 64)
    conv = g.he_probe_conversion_rate(8, 152, 64)
    recomb = g.he_probe_recombine_rate(152, 64)
    # GB300 at any clock: between 10^10 and 10^14 per second
    for r in (bfly, conv, recomb):
        assert 1e10 < r < 1e14, r
    for bad in ((0, 64), (152, 0), (152, 1 << 20)):
        with pytest.raises(g.HeError):
            g.he_probe_recombine_rate(*bad)
    with pytest.raises(g.HeError):
        g.he_probe_conversion_rate(3, 152, 64)
