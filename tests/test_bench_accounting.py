"""The benchmark's roofline accounting, checked on the CPU against independent
counts: the NTT passes' butterflies add up to the path's limb transforms, the
streaming kernels' bytes follow from the workspace layout, and every committed
profile line the benchmark reads parses and names an existing source.
"""
import glob
import os
import re

import pytest

import bench
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

NTT_KERNELS = ["intt_d2.inv_pass1", "intt_d2.inv_pass2", "ntt_modup.fwd_pass1", "ntt_modup.fwd_pass2",
               "intt_special.inv_pass1", "intt_special.inv_pass2", "ntt_moddown.fwd_pass1",
               "ntt_moddown.fwd_pass2_combine"]


@pytest.mark.parametrize("name,level,split", [("n16", 24, 0), ("n16", 9, 0), ("n17", 44, 0), ("n15", 16, 0),
                                              ("n16", 24, 1), ("n16", 24, 2), ("n17", 44, 1), ("n17", 44, 2)])
def test_ntt_butterflies_add_up_to_the_limb_transforms(name, level, split):
    prm = oracle.preset(name)
    N, K = prm.N, prm.K
    beta = -(-level // prm.alpha)
    # fused path: iNTT of d2 and the two last limbs of d0, d1; NTT of the ModUp
    # outputs (own-digit limbs reuse d2); iNTT of the 2K special limbs and the two
    # last KS limbs; NTT of the 2(l-1) ModDown limbs
    transforms = (level + 2) + (beta * (K + level) - level) + (2 * K + 2) + 2 * (level - 1)
    total = 0
    per = {}
    for k in NTT_KERNELS:
        kind, work = bench.kernel_work(k, prm, level, split)
        assert kind == "alu"
        total += work
        per[k] = work
    assert total == transforms * (N // 2) * prm.logN
    # the strided pass (first forward, second inverse) takes the split's stage count
    strided = {0: {16: 8, 17: 9}, 1: {16: 7, 17: 8}, 2: {16: 9, 17: 10}}[split].get(prm.logN)
    if strided is not None:
        assert per["ntt_modup.fwd_pass1"] == (beta * (K + level) - level) * (N // 2) * strided
        assert per["intt_special.inv_pass2"] == (2 * K + 2) * (N // 2) * strided
    if (name, level) == ("n16", 24):
        assert transforms == 162


@pytest.mark.parametrize("name,level", [("n16", 24), ("n17", 44)])
def test_streaming_and_conversion_work(name, level):
    prm = oracle.preset(name)
    N, K, alpha = prm.N, prm.K, prm.alpha
    beta = -(-level // alpha)
    E, limb = K + level, N * 8
    # inner product: U (beta E limbs, own rows from d2) and the key (2 beta E) read, KS (2E) written
    assert bench.kernel_work("inner_product", prm, level) == ("hbm", (beta * E + 2 * beta * E + 2 * E) * limb)
    # tensor: two ciphertexts (4l limbs) read, d0, d1, d2 (3l) written
    assert bench.kernel_work("tensor", prm, level) == ("hbm", 7 * level * limb)
    # ModUp: every digit j of n_j limbs converts to the E - n_j other limbs with n_j
    # inputs each (both levels here split into full digits: 24 = 3 x 8, 44 = 4 x 11)
    assert level % alpha == 0
    n_j = [min(alpha, level - j * alpha) for j in range(beta)]
    assert bench.kernel_work("modup", prm, level) == ("mac", sum(n * (E - n) for n in n_j) * N)
    assert bench.kernel_work("moddown_conv", prm, level) == ("mac", 2 * level * N * K)
    if (name, level) == ("n16", 24):
        assert bench.kernel_work("inner_product", prm, level)[1] == 184549376


def test_committed_profile_lines_parse():
    pat = re.compile(r"bench kernel: ([\w.]+) \| source (\S+) sha256 prefix ([0-9a-f]{16}) \| "
                     r"traffic_bytes_per_launch (\d+)")
    seen = {}
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        txt = open(path).read()
        for line in txt.splitlines():
            if line.startswith("bench kernel:"):
                m = pat.fullmatch(line.strip())
                assert m, (path, line)
                name, src, _, nbytes = m.groups()
                assert os.path.exists(os.path.join(ROOT, src)), src
                assert int(nbytes) > 0
                assert name not in seen, f"{name} in {path} and {seen.get(name)}"
                seen[name] = path
    # every kernel of the event profile of the fused step (the shape the
    # autotuner keeps at N = 2^16: tensor product and special rows' sums inside
    # their iNTTs, q rows beside the ModDown conversion) has a committed DRAM figure
    fused = ["intt_d2.tensor_inv_pass1"] + NTT_KERNELS[1:4] + ["intt_special.ip_inv_pass1"] + NTT_KERNELS[5:]
    for k in fused + ["modup", "moddown_conv_ipq"]:
        assert k in seen, k


@pytest.mark.parametrize("name,level,split", [("n16", 24, 1), ("n17", 44, 1), ("n16", 9, 0)])
def test_fused_and_onepass_profile_names(name, level, split):
    """The profile names of the fused and one-pass launches count the same
    butterflies as the plain passes they replace."""
    prm = oracle.preset(name)
    plain = bench.kernel_work("intt_special.inv_pass1", prm, level, split)
    assert bench.kernel_work("intt_special.ip_inv_pass1", prm, level, split) == plain
    assert bench.kernel_work("intt_d2.tensor_inv_pass1", prm, level, split) == \
        bench.kernel_work("intt_d2.inv_pass1", prm, level, split)
    for site in ("intt_d2", "ntt_modup", "intt_special", "ntt_moddown"):
        two = sum(bench.kernel_work(f"{site}.{d}_pass{k}", prm, level, split)[1]
                  for d in ("fwd", "inv") for k in (1, 2)) // 2
        kind, one = bench.kernel_work(f"{site}.{'fwd' if site.startswith('ntt') else 'inv'}_onepass", prm, level, split)
        assert kind == "alu" and one == two, site


def test_shape_dict_round_trip():
    t = (1, 8, 2, 15, 8, 7, 1, 1, 4, 0.25)
    d = bench.shape_dict(t)
    assert d == {"group_cap": 1, "modup_chunk": 8, "pdl": 2, "ntt_r8": 15, "ip_jobs": 8, "fuse": 7,
                 "ntt_split": 1, "ntt_small": 1, "ntt_onepass": 4, "ms": 0.25}
    assert "ms" not in bench.shape_dict(t[:9])
