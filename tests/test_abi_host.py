"""CPU-only checks of the library boundary: the shared library builds and
exports every symbol include/he.h declares; the host-side scheme functions
(parameters, key generation, encoding, encryption, decryption) agree with the
oracle on the same seeds; argument errors come back as status codes.
No GPU compute is run here.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import seeded_inputs as si
from oracle.encoding import encode

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def g():
    from paper_2003_04510_gb300 import build
    build.build()
    import paper_2003_04510_gb300 as pkg
    return pkg


def declared_functions():
    src = open(os.path.join(ROOT, "include", "he.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s*(he_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(g):
    names = declared_functions()
    assert len(names) >= 25
    lib = ctypes.CDLL(g.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    # and the binding wraps every one of them
    assert set(names) <= set(g._SIGS)


@pytest.mark.parametrize("name", ["n12", "n15", "n16", "n17"])
def test_params_match_oracle(g, name):
    ctx = g.Context(g.PRESETS[name][0], device=False)
    op = oracle.preset(name)
    assert np.array_equal(ctx.moduli, np.array(op.ext, dtype=np.uint64))
    assert ctx.dnum == op.dnum and ctx.N == op.N


def test_host_keygen_encrypt_match_oracle_n12(g):
    name = "n12"
    ctx = g.Context(g.PRESETS[name][0], device=False)
    op = oracle.preset(name)
    sc = 2.0 ** g.PRESETS[name][1]
    ks, s1, _ = si.SEEDS[name]
    sk, pk, evk = g.he_keygen(ctx, ks)
    osk = oracle.keygen_sk(op, ks)
    assert np.array_equal(sk, osk)
    assert np.array_equal(pk, oracle.keygen_pk(op, osk, ks))
    assert np.array_equal(evk, oracle.keygen_evk(op, osk, ks))
    m = si.messages(op.N // 2, s1)
    pt_o = encode(m, op.logN, sc)
    pt_g = g.he_encode(ctx, m, sc)
    # two FFTs round the same reals: allow a unit difference where they straddle .5
    assert np.abs(pt_o - pt_g).max() <= 1
    for level in (3, 2, 1):
        ct_g = g.he_encrypt_poly(ctx, pk, pt_o, level, s1 + level)
        ct_o = oracle.encrypt_poly(op, pk, pt_o, level, s1 + level)
        assert np.array_equal(ct_g, ct_o)
        assert np.array_equal(g.he_decrypt_poly(ctx, sk, ct_g, level), oracle.decrypt_residues(op, sk, ct_o, level))
    z = g.he_decrypt(ctx, sk, g.he_encrypt(ctx, pk, m, sc, 3, 5), 3, sc)
    assert np.abs(z - m).max() < 2.0 ** -20
    zz = g.he_decode(ctx, g.he_encode(ctx, m, sc).astype(np.float64) / sc)
    assert np.abs(zz - m).max() < 2.0 ** -30


def test_host_keygen_matches_oracle_n15(g):
    name = "n15"
    ctx = g.Context(g.PRESETS[name][0], device=False)
    op = oracle.preset(name)
    ks = si.SEEDS[name][0]
    sk, pk, _ = g.he_keygen(ctx, ks)
    osk = oracle.keygen_sk(op, ks)
    assert np.array_equal(sk, osk)
    assert np.array_equal(pk, oracle.keygen_pk(op, osk, ks))


def test_host_rotation_keys_match_oracle_n12(g):
    name = "n12"
    ctx = g.Context(g.PRESETS[name][0], device=False)
    op = oracle.preset(name)
    sk = oracle.keygen_sk(op, si.SEEDS[name][0])
    for steps in (1, -1, 7, op.N // 2 + 3):
        gl = g.he_galois_elt(ctx, steps)
        assert gl == oracle.galois_elt(op, steps)
        assert np.array_equal(g.he_keygen_rot(ctx, 77, sk, gl), oracle.keygen_rot(op, sk, gl, 77))
    gc = g.he_conj_elt(ctx)
    assert gc == oracle.conj_elt(op)
    assert np.array_equal(g.he_keygen_rot(ctx, 78, sk, gc), oracle.keygen_rot(op, sk, gc, 78))
    for bad in (0, 2, 2 * op.N, 2 * op.N + 1):
        with pytest.raises(g.HeError) as e:
            g.he_keygen_rot(ctx, 1, sk, bad)
        assert e.value.code == g.HE_EINVAL


def test_host_plaintext_ntt_matches_oracle(g):
    for name in ("n12", "n16"):
        ctx = g.Context(g.PRESETS[name][0], device=False)
        op = oracle.preset(name)
        rng = np.random.default_rng(5)
        t = rng.integers(-(1 << 62), 1 << 62, size=op.N, dtype=np.int64)
        t[0] = np.iinfo(np.int64).min
        t[1] = np.iinfo(np.int64).max
        for level in (op.L, 1):
            assert np.array_equal(g.he_plain_ntt(ctx, t, level), oracle.plain_ntt(op, t, level))


def test_host_seeded_key_matches_oracle_n12(g):
    name = "n12"
    ctx = g.Context(g.PRESETS[name][0], device=False)
    op = oracle.preset(name)
    sk = oracle.keygen_sk(op, si.SEEDS[name][0])
    full = oracle.keygen_evk_seeded(op, sk, 4242)
    assert np.array_equal(g.he_keygen_seeded(ctx, 4242, sk), full[:, 0])


def test_shape_setters(g):
    ctx = g.Context(g.PRESETS["n12"][0], device=False)
    assert g.he_get_shape(ctx) == (4, 8, 1, 0, 8, 7, 0, 0, 0)
    g.he_set_shape(ctx, 2, 16, 0)
    assert g.he_get_shape(ctx) == (2, 16, 0, 0, 8, 7, 0, 0, 0)
    g.he_set_shape(ctx, 2, 16, 0, 5, 4, 0)
    assert g.he_get_shape(ctx) == (2, 16, 0, 5, 4, 0, 0, 0, 0)
    g.he_set_shape(ctx, 2, 16, 2, 5, 4, 0, 2, 9)
    assert g.he_get_shape(ctx) == (2, 16, 2, 5, 4, 0, 2, 9, 0)
    g.he_set_shape(ctx, 2, 16, 2, 5, 4, 0, 2, 9, 6)
    assert g.he_get_shape(ctx) == (2, 16, 2, 5, 4, 0, 2, 9, 6)
    g.he_set_shape(ctx, 2, 16, 0, 5, 4, 0)
    for bad in ((0, 8, 1, 0, 8, 1), (5, 8, 1, 0, 8, 1), (4, 6, 1, 0, 8, 1), (4, 32, 1, 0, 8, 1), (4, 8, 3, 0, 8, 1),
                (4, 8, -1, 0, 8, 1),
                (4, 8, 1, 16, 8, 1), (4, 8, 1, -1, 8, 1), (4, 8, 1, 0, 0, 1), (4, 8, 1, 0, 2, 1), (4, 8, 1, 0, 9, 1),
                (4, 8, 1, 0, 8, 8), (4, 8, 1, 0, 8, -1), (4, 8, 1, 0, 8, 1, 3), (4, 8, 1, 0, 8, 1, -1),
                (4, 8, 1, 0, 8, 1, 0, 16), (4, 8, 1, 0, 8, 1, 0, -1), (4, 8, 1, 0, 8, 1, 0, 0, 16),
                (4, 8, 1, 0, 8, 1, 0, 0, -1)):
        with pytest.raises(g.HeError) as e:
            g.he_set_shape(ctx, *bad)
        assert e.value.code == g.HE_EINVAL
    assert g.he_get_shape(ctx) == (2, 16, 0, 5, 4, 0, 0, 0, 0)


def test_argument_errors_are_status_codes(g):
    bad = g.Params(11, 3, 1, 1, 50, 51, 64)  # logN below range
    with pytest.raises(g.HeError) as e:
        g.Context(bad, device=False)
    assert e.value.code == g.HE_EINVAL
    with pytest.raises(g.HeError):
        g.Context(g.Params(12, 3, 1, 1, 58, 51, 64), device=False)  # primes too wide
    ctx = g.Context(g.PRESETS["n12"][0], device=False)
    # device entry points refuse a host-only context before touching CUDA
    rc = g.lib().he_mul(ctx.ptr, 256, 256, 256, 3, 256, 256, 1 << 30, None)
    assert rc == g.HE_EINVAL
    assert g.lib().he_workspace_bytes(ctx.ptr, 0) == 0
    assert g.lib().he_workspace_bytes(ctx.ptr, 4) == 0
    assert g.lib().he_workspace_bytes(ctx.ptr, 3) > 0
    with pytest.raises(g.HeError) as e:
        g.he_encrypt_poly(ctx, np.zeros((2, 3, 4096), np.uint64), np.zeros(4096, np.int64), 4, 1)
    assert e.value.code == g.HE_ELEVEL
    assert g.lib().he_strerror(g.HE_ETIMEOUT) == b"bounded device wait gave up"


def test_probe_argument_errors_need_no_gpu(g):
    """The probes check their arguments before any CUDA call."""
    st = 0  # a stream handle the calls never reach
    for call in (lambda: g.he_probe_recombine_rate(0, 64, st), lambda: g.he_probe_recombine_rate(152, 0, st),
                 lambda: g.he_probe_recombine_rate(152, 1 << 20, st),
                 lambda: g.he_probe_conversion_rate(3, 152, 64, st), lambda: g.he_probe_conversion_rate(8, 0, 64, st),
                 lambda: g.he_probe_butterfly_rate(0, 64, st)):
        with pytest.raises(g.HeError) as e:
            call()
        assert e.value.code == g.HE_EINVAL
