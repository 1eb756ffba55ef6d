"""Benchmark: HE Mul + relinearise + rescale throughput on GB300.

Default workload (N=1): one HE Mul of two fresh ciphertexts at N = 2^16,
24 x 54-bit limbs + 8 x 55-bit special primes, dnum 3, level 24 -> 23 after
rescale (he_mul_rescale, bit-identical to he_mul followed by he_rescale).
A step is one HE Mul + rescale of one ciphertext pair.  Eight distinct pairs
are rotated so that the step's inputs (pairs + evaluation key, 480 MB) exceed
the 129 MB L2.

Printed JSON line (rank 0):
  value       HE Mul/s with inputs resident in HBM (CUDA events on the stream)
  e2e         HE Mul/s through he_mul_rescale_host: host->device copy of both
              operands, the path, device->host copy of the result, per step
  latency     p50 / p99 per-step device latency (ms)
  roofline    the dominant kernel of the event profile against its ceiling:
              NTT passes in butterflies/s against the measured butterfly probe
              (the NTT's own butterfly), base conversions in MACs/s against the
              measured conversion probe (their own inner loop), streaming
              kernels in GB/s against the measured HBM copy rate
  cpu_baseline  the CPU oracle on the host cores, bounded sample
  clocks      SM clocks sampled with nvidia-smi during the timed region

--impl reference times the CPU oracle (the deliberately plain C checker) on
the same workload as the reference arm.  With torchrun (N>1) every rank runs
its own independent HE Muls on its own GPU (weak scaling, no collective on the
data path); the reported time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import seeded_inputs as si  # noqa: E402

WORKLOADS = {
    # name: (preset, level, description)
    "n16": ("n16", 24, "single HE Mul+relin+rescale, N=2^16, 24x54-bit limbs + 8x55-bit specials, dnum 3, level 24->23"),
    "n17": ("n17", 44, "single HE Mul+relin+rescale, N=2^17, 44x54-bit limbs + 12x54-bit specials, dnum 4, level 44->43"),
    "n12": ("n12", 3, "single HE Mul+relin+rescale, N=2^12, 3x50-bit limbs + 1x51-bit special, alpha 1, level 3->2"),
}
NPAIRS = 8


def reduce_max(x: float, device=None) -> float:
    """Max of a per-rank float over all ranks (no-op without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, world: int, max_seconds: float) -> float:
    """Whole-job throughput: units processed by all ranks over the slowest rank's time."""
    return world * units_per_rank / max_seconds


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms in the background."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------
def oracle_inputs(preset: str, level: int):
    import oracle
    from oracle.encoding import encode
    op = oracle.preset(preset)
    sc = 2.0 ** oracle.PRESETS[preset]["scale_bits"]
    ks, s1, s2 = si.SEEDS[preset]
    sk = oracle.keygen_sk(op, ks)
    pk = oracle.keygen_pk(op, sk, ks)
    evk = oracle.keygen_evk(op, sk, ks)
    m1, m2 = si.messages(op.N // 2, s1), si.messages(op.N // 2, s2)
    ct1 = oracle.encrypt_poly(op, pk, encode(m1, op.logN, sc), level, s1)
    ct2 = oracle.encrypt_poly(op, pk, encode(m2, op.logN, sc), level, s2)
    return op, ct1, ct2, evk


def time_oracle(preset: str, level: int, budget_s: float, max_steps: int | None = None):
    """Oracle HE Mul + rescale repeated until budget_s is spent (at least once)."""
    import oracle
    op, ct1, ct2, evk = oracle_inputs(preset, level)
    times = []
    t_all = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        c3 = oracle.he_mul(op, ct1, ct2, evk, level)
        oracle.rescale(op, c3, level)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_all >= budget_s or (max_steps and len(times) >= max_steps):
            break
    return times


def _oracle_worker(job):
    preset, level, budget_s, max_steps = job
    t = time_oracle(preset, level, budget_s, max_steps)
    return len(t), float(sum(t))


def time_oracle_cores(preset: str, level: int, budget_s: float, procs: int, max_steps: int | None = None):
    """The unmodified single-threaded oracle run as `procs` independent processes
    (one HE Mul stream per host core, the data-parallel shape of the workload).
    Returns (aggregate HE Mul/s, HE Muls done, per-process rates).  The pool is
    started with spawn, so it is safe after CUDA has been initialised."""
    import multiprocessing as mp
    per = None if max_steps is None else max(1, -(-max_steps // procs))
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_oracle_worker, [(preset, level, budget_s, per)] * procs)
    rates = [n / t for n, t in res]
    return float(sum(rates)), int(sum(n for n, _ in res)), rates


def host_cores() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except Exception:
        return max(1, os.cpu_count() or 1)


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    preset, level, desc = WORKLOADS[args.workload]
    # the sample is bounded by time: every host core runs the plain oracle
    # on its own HE Muls for about HE_REF_BUDGET_S seconds
    budget = float(os.environ.get("HE_REF_BUDGET_S", "60"))
    cores = host_cores()
    value, done, rates = time_oracle_cores(preset, level, budget, cores, max_steps=args.steps)
    line = {
        "impl": "reference", "metric": "HE Mul/s (HE Mul + relinearize + rescale)", "value": value,
        "unit": "HE Mul/s", "n_gpus": args.gpus, "steps": done, "warmup": 0,
        "ms_per_step": 1e3 / value, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic (seeded encryptions of unit-disk messages)",
        "config": {"workload": desc},
        "cpu_baseline": {"value": value, "unit": "HE Mul/s", "cores": cores, "kind": "oracle",
                         "sample": f"{done} full HE Mul+rescale runs of the plain single-threaded oracle, one "
                                   f"process per host core ({cores}), ~{budget:.0f} s each (of {args.steps} "
                                   f"requested)",
                         "single_core_value": min(rates)},
        "e2e": {"value": value, "unit": "HE Mul/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
# stages of the strided pass under the launch shape's NTT pass split (1, 2) at
# the ring sizes that have one; the contiguous pass takes the rest
SPLIT_STRIDED = {(16, 1): 7, (16, 2): 9, (17, 1): 8, (17, 2): 10}


def kernel_work(name: str, prm, level: int, split: int = 0):
    """Algorithmic work of one launch of kernel `name` at this level:
    ("alu", butterflies) for NTT passes, ("hbm", bytes) for the streaming kernels.
    `split` is the launch shape's NTT pass split (stages per pass)."""
    N, K, alpha = 1 << prm.logN, prm.K, prm.alpha
    beta = -(-level // alpha)
    E = K + level
    limb = N * 8
    passes = {16: (8, 8), 17: (9, 8), 15: (8, 7), 14: (7, 7), 13: (7, 6), 12: (12, 0)}[prm.logN]
    if (prm.logN, split) in SPLIT_STRIDED:
        passes = (SPLIT_STRIDED[(prm.logN, split)], prm.logN - SPLIT_STRIDED[(prm.logN, split)])
    jobs = {"intt_d2": level + 2, "ntt_modup": beta * E - level, "intt_special": 2 * K + 2,
            "ntt_moddown": 2 * (level - 1)}
    base = name.split(".")[0]
    if base in jobs:
        fwd = ".fwd" in name
        if prm.logN == 12 or "onepass" in name:
            stages = prm.logN
        elif fwd:
            stages = passes[0] if name.endswith("pass1") else passes[1]
        else:
            stages = passes[1] if name.endswith("pass1") else passes[0]
        return "alu", jobs[base] * (N // 2) * stages
    if base == "inner_product":
        return "hbm", (3 * beta + 2) * E * limb
    if base == "inner_product_special":  # the special limbs and q_{l-1}
        return "hbm", (3 * beta + 2) * (K + 1) * limb
    if base == "moddown_conv_ipq":  # conversion (ALU) and the q limbs' key-switch sums (HBM) in one launch
        return "mixed", 2 * level * N * K
    if base == "tensor":
        return "hbm", 7 * level * limb
    if base == "modup":  # 64x64-bit multiply-accumulates
        return "mac", (beta * E - level) * N * alpha
    if base == "moddown_conv":
        return "mac", 2 * level * N * K
    if base == "combine_rescale":
        return "hbm", (2 * level + 2 * level + 2 * (level - 1) + 2 * (level - 1)) * limb
    return None, 0


def kernel_width(n: int) -> int:
    """The padded term count a conversion kernel is instantiated for (1, 2, 4, 8, 12, 16)."""
    return next(w for w in (1, 2, 4, 8, 12, 16) if w >= n)


def shape_dict(t) -> dict:
    """A launch shape (group_cap, modup_chunk, pdl, ntt_r8, ip_jobs, fuse, ntt_split, ntt_small, ntt_onepass[, ms])
    as a dict."""
    d = dict(zip(("group_cap", "modup_chunk", "pdl", "ntt_r8", "ip_jobs", "fuse", "ntt_split", "ntt_small",
                  "ntt_onepass"), t[:9]))
    if len(t) > 9:
        d["ms"] = t[9]
    return d


def committed_traffic(kernel: str):
    """Per-launch DRAM bytes of `kernel` (a name of the bench's event profile)
    from a committed ncu summary under profiles/ that names it ("bench kernel:
    <name>") with "traffic_bytes_per_launch | <bytes>", or None when no summary
    covers it or the source file it names changed after the capture (sha256
    prefix)."""
    import glob
    import hashlib
    import re
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        txt = open(path).read()
        for m in re.finditer(r"bench kernel: ([\w.]+) \| source (\S+) sha256 prefix ([0-9a-f]{16}) \| "
                             r"traffic_bytes_per_launch (\d+)", txt):
            if m.group(1) != kernel:
                continue
            src = os.path.join(ROOT, m.group(2))
            if not os.path.exists(src):
                return None
            if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != m.group(3):
                return None
            return int(m.group(4))
    return None


def hbm_peak_gbs() -> float:
    """The measured HBM copy rate (MEASURED_PEAKS.json), else the fallback."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0))
    except Exception:
        return 6800.0


def inner_product_alone(g, ctx, step, level, steps=10):
    """The key-switch inner product as its own kernel (all K + l rows; the
    shape's split and fused-sum bits off and programmatic launch off for these
    steps only, so no neighbouring kernel shares its SMs), timed in the event
    profile: its HBM rate against the measured copy rate.  With the autotuned
    shape the same sums run inside the ModDown launch and the special limbs'
    first iNTT pass, where no kernel has them alone."""
    shape = g.he_get_shape(ctx)
    g.he_set_shape(ctx, *(shape[:2] + (0,) + shape[3:5] + (shape[5] & 1,) + shape[6:]))
    try:
        for k in range(3):
            step(k)
        g.he_profile(ctx, True)
        for k in range(steps):
            step(k)
        prof = g.he_profile_read(ctx)
        g.he_profile(ctx, False)
    finally:
        g.he_set_shape(ctx, *shape)
    if "inner_product" not in prof:
        return None
    us = prof["inner_product"][0] / prof["inner_product"][1] * 1e3
    _, b = kernel_work("inner_product", ctx.prm, level)
    ach = b / (us * 1e-6) / 1e9
    peak = hbm_peak_gbs()
    return {"us": us, "bytes": b, "achieved_gbs": ach, "peak_gbs": peak, "frac": ach / peak,
            "what": "the inner product with the evaluation key (all rows) as its own kernel, no programmatic "
                    "launch, same shape otherwise"}


def run_batched(g, ctx, evk_t, dev, stream, wsz, count=64, reps=20):
    """64 independent HE Mul + rescale jobs, levels uniform in 4..24 (seeded),
    operands uniform residues (same bytes and work as encryptions), as one
    he_mul_batch versus the same jobs issued one he_mul_rescale at a time."""
    import torch
    levels = [int(v) for v in si.batch_levels(count, 4, 24)]
    N = ctx.N
    jobs = []
    for k, lv in enumerate(levels):
        q = [int(x) for x in ctx.q[:lv]]
        a = np.stack([si.uniform_residues(q, (N,), 7000 + 4 * k + h) for h in range(2)])
        b = np.stack([si.uniform_residues(q, (N,), 7002 + 4 * k + h) for h in range(2)])
        out = torch.empty((2, lv - 1, N), dtype=torch.int64, device=dev)
        jobs.append((g.to_device(a, dev), g.to_device(b, dev), out, lv))
    wsb = torch.empty(g.he_batch_workspace_bytes(ctx, levels) // 8, dtype=torch.int64, device=dev)
    ws1 = g.workspace(ctx, max(levels), device=dev)
    # launch shapes picked by the library's autotuner on this very batch
    shape_before = g.he_get_shape(ctx)
    best, tried = g.he_autotune(ctx, jobs, evk_t, wsb, reps=3, stream=stream)

    def batch():
        g.he_mul_batch(ctx, jobs, evk_t, wsb, stream)

    def singles():
        for a, b, o, lv in jobs:
            g.he_mul_rescale(ctx, a, b, evk_t, lv, o, ws1, stream)

    graph = g.BatchGraph(ctx, count, evk_t, stream, device=dev)

    def graphed():
        graph.launch(jobs, stream)

    res = {}
    for name, fn in (("batched", batch), ("batched_graph", graphed), ("single_path", singles)):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        # the timed loop three times (a host stall in one does not set the
        # figure): the median of the three totals
        totals, lat = [], []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
            e0.record(stream)
            for r in range(reps):
                ev[r][0].record(stream)
                fn()
                ev[r][1].record(stream)
            e1.record(stream)
            torch.cuda.synchronize()
            totals.append(e0.elapsed_time(e1))
            lat += [a.elapsed_time(b) for a, b in ev]
        ms = float(np.median(totals))
        lat = np.array(lat)
        res[name] = {"HE_Mul_per_s": wsz * count * reps / (ms * 1e-3), "ms_per_batch": ms / reps,
                     "loops_ms": totals, "batch_latency_ms_p50": float(np.percentile(lat, 50)),
                     "batch_latency_ms_p99": float(np.percentile(lat, 99))}
    graph.close()
    # per-kernel device time of one batch (CUDA events between the launches)
    g.he_profile(ctx, True)
    for _ in range(5):
        batch()
    prof = g.he_profile_read(ctx)
    g.he_profile(ctx, False)
    res["kernels_us"] = {k: v[0] / v[1] * 1e3 for k, v in prof.items()}
    if "inner_product" in prof:
        ip_bytes = sum(kernel_work("inner_product", ctx.prm, lv)[1] for lv in levels)
        res["inner_product_gbs"] = ip_bytes / (res["kernels_us"]["inner_product"] * 1e-6) / 1e9
    g.he_set_shape(ctx, *shape_before)
    res["autotune"] = dict(shape_dict(best), ms_per_batch=best[9], tried=[shape_dict(t) for t in tried])
    res["config"] = {"jobs": count, "N": N, "levels": "uniform 4..24 (seed 1604)", "mean_level": float(np.mean(levels)),
                     "operands": "uniform residues"}
    return res


def run_serving(g, dev, rate_hz=2000.0, duration_s=10.0, streams=4, max_batch=64):
    """Poisson stream of HE Mul + rescale requests: 70% N=2^15 (levels 2..16),
    30% N=2^16 (levels 4..24), both rings' evaluation keys resident; operands
    are uniform residues (one pair per ring and level), outputs rotate over a
    pool.  Reports throughput and p50/p99 latency (submit -> completion)."""
    import torch
    rings = ["n15", "n16"]
    ctxs = [g.Context(g.PRESETS[r][0], device=True) for r in rings]
    evks, pairs, pools = [], [], []
    for ri, ctx in enumerate(ctxs):
        ext = [int(x) for x in ctx.moduli]
        evk = np.stack([np.stack([si.uniform_residues(ext, (ctx.N,), 9000 + 10 * ri + 2 * j + h) for h in range(2)])
                        for j in range(ctx.dnum)])
        evks.append(g.to_device(evk, dev))
        pr = {}
        lo, hi = (2, 16) if ri == 0 else (4, 24)
        for lv in range(lo, hi + 1):
            q = [int(x) for x in ctx.q[:lv]]
            pr[lv] = tuple(g.to_device(np.stack([si.uniform_residues(q, (ctx.N,), 9500 + 100 * ri + 4 * lv + 2 * k + h)
                                                  for h in range(2)]), dev) for k in range(2))
        pairs.append(pr)
        L = ctx.prm.L
        pools.append(torch.empty((256, 2 * (L - 1) * ctx.N), dtype=torch.int64, device=dev))
    arrivals = si.poisson_arrivals(rate_hz, duration_s)
    mix = si.serving_mix(len(arrivals))
    budget = 16 << 30
    # warm-up on a throwaway server: one request per ring and level, so that
    # first-use costs (kernel loading, the stream-ordered allocator's pool)
    # fall outside the measured stream
    warm = g.Server(ctxs, evks, hbm_budget=budget, max_batch=max_batch, streams=streams)
    for ri, ctx in enumerate(ctxs):
        for lv, (a, b) in pairs[ri].items():
            warm.wait(warm.submit(ri, lv, a, b, pools[ri][lv][: 2 * (lv - 1) * ctx.N]), 600000)
    warm.close()
    srv = g.Server(ctxs, evks, hbm_budget=budget, max_batch=max_batch, streams=streams)
    tickets = []
    t0 = time.perf_counter()
    for k, (ta, (logN, lv)) in enumerate(zip(arrivals, mix)):
        ri = 0 if logN == 15 else 1
        while time.perf_counter() - t0 < ta:
            pass
        a, b = pairs[ri][lv]
        out = pools[ri][k % 256][: 2 * (lv - 1) * ctxs[ri].N]
        tickets.append(srv.submit(ri, lv, a, b, out))
    for tk in tickets:
        srv.wait(tk, 600000)
    st = srv.stats()
    srv.close()
    return {"requests": len(tickets), "rate_hz": rate_hz, "duration_s": duration_s,
            "throughput_req_s": st["throughput"], "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
            "max_ms": st["max_ms"], "batches": st["batches"], "mean_batch": st["mean_batch"],
            "mix": "70% N=2^15 levels 2..16, 30% N=2^16 levels 4..24", "streams": streams, "max_batch": max_batch,
            "hbm_budget_bytes": budget}


def run_single(g, preset, level, dev, stream, rank, reps=300, npairs=2):
    """Single HE Mul + rescale at another ring size (N = 2^17 beside the
    default 2^16): autotuned shape, per-step latency, per-kernel profile and
    the inner product's HBM fraction."""
    import torch
    prm, scale_bits = g.PRESETS[preset]
    sc = 2.0 ** scale_bits
    ctx = g.Context(prm, device=True)
    N = ctx.N
    ks, s1, s2 = si.SEEDS[preset]
    sk, pk, evk = g.he_keygen(ctx, ks + 1000 * rank)
    evk_t = g.to_device(evk, dev)
    del evk
    ct_t = [(g.to_device(g.he_encrypt(ctx, pk, si.messages(N // 2, s1 + 17 * k), sc, level, s1 + 17 * k), dev),
             g.to_device(g.he_encrypt(ctx, pk, si.messages(N // 2, s2 + 17 * k), sc, level, s2 + 17 * k), dev))
            for k in range(npairs)]
    outs = [torch.empty((2, level - 1, N), dtype=torch.int64, device=dev) for _ in range(npairs)]
    ws = g.workspace(ctx, level, device=dev)
    best, _ = g.he_autotune(ctx, [(ct_t[0][0], ct_t[0][1], outs[0], level)], evk_t, ws, reps=10, stream=stream)

    def step(k):
        a, b = ct_t[k % npairs]
        g.he_mul_rescale(ctx, a, b, evk_t, level, outs[k % npairs], ws, stream)

    for k in range(5):
        step(k)
    torch.cuda.synchronize()
    z = g.he_decrypt(ctx, sk, g.to_host(outs[0]), level - 1, sc * sc / float(ctx.q[level - 1]))
    err = float(np.abs(z - si.messages(N // 2, s1) * si.messages(N // 2, s2)).max())
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    for k in range(reps):
        step(k)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / reps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for k in range(reps):
        ev[k][0].record(stream)
        step(k)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    lat = np.array([a.elapsed_time(b) for a, b in ev])
    g.he_profile(ctx, True)
    for k in range(10):
        step(k)
    prof = g.he_profile_read(ctx)
    g.he_profile(ctx, False)
    kernels_us = {k: v[0] / v[1] * 1e3 for k, v in prof.items()}
    ip = inner_product_alone(g, ctx, step, level)
    res = {"workload": WORKLOADS[preset][2], "HE_Mul_per_s": 1e3 / ms, "ms": ms, "reps": reps,
           "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
           "autotune": shape_dict(best),
           "kernels_us": kernels_us, "inner_product_hbm": ip,
           "evk_bytes": int(evk_t.numel() * 8), "decrypt_max_err": err,
           "l2": f"{npairs} ciphertext pairs + evk rotated "
                 f"({(npairs * 4 * level + 2 * ctx.dnum * (prm.K + prm.L)) * N * 8 / 1e6:.0f} MB > 129 MB L2)"}
    del ws, outs, ct_t, evk_t
    ctx.close()
    return res


def run_ours(args):
    import torch
    import paper_2003_04510_gb300 as g
    from paper_2003_04510_gb300 import build as gb

    wsz, rank, local = dist_env()
    if wsz > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    gb.build()

    preset, level, desc = WORKLOADS[args.workload]
    prm, scale_bits = g.PRESETS[preset]
    sc = 2.0 ** scale_bits
    ctx = g.Context(prm, device=True)
    N = ctx.N
    ks, s1, s2 = si.SEEDS[preset]
    sk, pk, evk = g.he_keygen(ctx, ks + 1000 * rank)
    pairs = []
    for k in range(NPAIRS):
        m1 = si.messages(N // 2, s1 + 17 * k)
        m2 = si.messages(N // 2, s2 + 17 * k)
        c1 = g.he_encrypt(ctx, pk, m1, sc, level, s1 + 17 * k)
        c2 = g.he_encrypt(ctx, pk, m2, sc, level, s2 + 17 * k)
        pairs.append((c1, c2))
    evk_t = g.to_device(evk, dev)
    ct_t = [(g.to_device(a, dev), g.to_device(b, dev)) for a, b in pairs]
    outs = [torch.empty((2, level - 1, N), dtype=torch.int64, device=dev) for _ in range(NPAIRS)]
    ws = g.workspace(ctx, level, device=dev)
    stream = torch.cuda.current_stream()

    def step(k):
        a, b = ct_t[k % NPAIRS]
        g.he_mul_rescale(ctx, a, b, evk_t, level, outs[k % NPAIRS], ws, stream)

    # launch shapes picked by the library's autotuner for this single HE Mul
    # (or fixed by --shape, e.g. for a profiler run)
    if args.shape:
        given = [int(v) for v in args.shape.split(",")]
        shape = (given + [0, 8, 7, 0, 0, 0][len(given) - 3:])[:9]
        g.he_set_shape(ctx, *shape)
        tune_best, tune_tried = tuple(shape) + (0.0,), []
    else:
        tune_best, tune_tried = g.he_autotune(ctx, [(ct_t[0][0], ct_t[0][1], outs[0], level)], evk_t, ws, reps=20,
                                              stream=stream)
    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()

    # correctness guard on the measured configuration: decrypt one result
    z = g.he_decrypt(ctx, sk, g.to_host(outs[0]), level - 1, sc * sc / float(ctx.q[level - 1]))
    m_exp = si.messages(N // 2, s1) * si.messages(N // 2, s2)
    dec_err = float(np.abs(z - m_exp).max())

    # ---- timed region: inputs resident in HBM; events only at its two ends
    # (an event between steps would stop the next step's first kernel from
    # overlapping the previous step's last one) ----
    clocks = ClockSampler(local)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    if wsz > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    t0.record(stream)
    for k in range(args.steps):
        step(k)
    t1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if wsz > 1:
        torch.distributed.barrier()
    elapsed_ms = reduce_max(t0.elapsed_time(t1), dev)
    # the same K-step region repeated: its spread says how steady the first is
    rep_ms = [elapsed_ms]
    for _ in range(4):
        if wsz > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0.record(stream)
        for k in range(args.steps):
            step(k)
        t1.record(stream)
        torch.cuda.synchronize()
        rep_ms.append(reduce_max(t0.elapsed_time(t1), dev))
    # per-step latency: a separate pass, each step between its own two events
    lat_steps = max(10, min(args.steps, 1000))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(lat_steps)]
    for k in range(lat_steps):
        ev[k][0].record(stream)
        step(k)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    lat = np.array([a.elapsed_time(b) for a, b in ev])
    value = job_rate(args.steps, wsz, elapsed_ms * 1e-3)
    # the final combine runs inside the last NTT pass; with fuse bit 0 the
    # tensor product runs inside the first one (bit 1 moves the q rows of the
    # inner product into the ModDown launch: the launch count stays; bit 2
    # with it moves the other rows into the special limbs' iNTT: one fewer)
    fz = g.he_get_shape(ctx)[5]
    launches_per_step = (12 if prm.logN > 12 else 8) - (1 if fz & 1 else 0) - (1 if (fz & 6) == 6 else 0)

    # ---- end to end: host buffers through he_mul_rescale_host ----
    hws = torch.empty(g.he_host_workspace_bytes(ctx, level) // 8, dtype=torch.int64, device=dev)
    pin = [(torch.from_numpy(a.view(np.int64)).pin_memory(), torch.from_numpy(b.view(np.int64)).pin_memory())
           for a, b in pairs[:2]]
    pin_out = torch.empty((2, level - 1, N), dtype=torch.int64).pin_memory()
    pin_np = [(a.numpy().view(np.uint64), b.numpy().view(np.uint64)) for a, b in pin]
    out_np = pin_out.numpy().view(np.uint64)
    # one synchronous call per step (upload, path, download, wait)
    single_steps = max(3, min(args.steps, 20))
    for k in range(2):
        a, b = pin_np[k % 2]
        g.he_mul_rescale_host(ctx, a, b, evk_t, level, out_np, hws, stream)
    torch.cuda.synchronize()
    te = time.perf_counter()
    for k in range(single_steps):
        a, b = pin_np[k % 2]
        g.he_mul_rescale_host(ctx, a, b, evk_t, level, out_np, hws, stream)
    single_val = single_steps / (time.perf_counter() - te)
    # the pipelined stream of host jobs: each step still uploads its operands
    # and downloads its result, overlapped with the neighbouring steps' kernels
    slots = 3
    sws = torch.empty(g.he_host_stream_workspace_bytes(ctx, level, slots) // 8, dtype=torch.int64, device=dev)
    e2e_steps = 200  # fixed, independent of --steps: a few tenths of a second of host wall clock per run
    s_ct1 = [pin_np[k % 2][0] for k in range(e2e_steps)]
    s_ct2 = [pin_np[k % 2][1] for k in range(e2e_steps)]
    g.he_mul_rescale_host_stream(ctx, s_ct1[:4], s_ct2[:4], [level] * 4, [out_np] * 4, evk_t, sws, slots, stream)
    if wsz > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e2e_runs = []
    for _ in range(3):
        if wsz > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        te = time.perf_counter()
        g.he_mul_rescale_host_stream(ctx, s_ct1, s_ct2, [level] * e2e_steps, [out_np] * e2e_steps, evk_t, sws,
                                     slots, stream)
        e2e_runs.append(job_rate(e2e_steps, wsz, reduce_max(time.perf_counter() - te, dev)))
    e2e_val = float(np.median(e2e_runs))
    zs = g.he_decrypt(ctx, sk, out_np, level - 1, sc * sc / float(ctx.q[level - 1]))
    m_last = si.messages(N // 2, s1 + 17 * ((e2e_steps - 1) % 2)) * si.messages(N // 2, s2 + 17 * ((e2e_steps - 1) % 2))
    e2e_err = float(np.abs(zs - m_last).max())
    del sws
    h2d = 2 * 2 * level * N * 8
    d2h = 2 * (level - 1) * N * 8
    # the host link's bound on the same bytes: each step's two uploads and one
    # download as plain copies (no kernels), on three streams as the host
    # stream issues them (one per operand upload, one for the download)
    link_steps = 100
    lin = torch.empty((2, 2 * level * N), dtype=torch.int64, device=dev)
    lout = torch.empty_like(pin_out, device=dev)
    sts = [torch.cuda.Stream(device=dev) for _ in range(3)]
    torch.cuda.synchronize()
    te = time.perf_counter()
    for k in range(link_steps):
        for h in range(2):
            with torch.cuda.stream(sts[h]):
                lin[h].copy_(pin[k % 2][h].view(-1), non_blocking=True)
        with torch.cuda.stream(sts[2]):
            pin_out.copy_(lout, non_blocking=True)
    torch.cuda.synchronize()
    link_val = link_steps / (time.perf_counter() - te)
    del lin, lout

    # ---- per-kernel profile (CUDA events on the launch stream) ----
    g.he_profile(ctx, True)
    prof_steps = min(args.steps, 20)
    for k in range(prof_steps):
        step(k)
    prof = g.he_profile_read(ctx)
    g.he_profile(ctx, False)
    per_kernel = {}
    split = g.he_get_shape(ctx)[6]
    for k, v in prof.items():
        kind, work = kernel_work(k, ctx.prm, level, split)
        d = {"ms_total": v[0], "calls": v[1], "ms_avg": v[0] / v[1], "kind": kind}
        if kind == "alu":
            d["Gbutterfly_s"] = work / (d["ms_avg"] * 1e-3) / 1e9
        elif kind == "hbm":
            d["GB_s"] = work / (d["ms_avg"] * 1e-3) / 1e9
        elif kind == "mac":
            d["GMAC_s"] = work / (d["ms_avg"] * 1e-3) / 1e9
        per_kernel[k] = d
    # the dominant kernel with one roofline (a launch mixing a compute-bound and
    # a memory-bound part has neither)
    graded = [k for k in per_kernel if per_kernel[k]["kind"] in ("alu", "mac", "hbm")]
    dom = max(graded, key=lambda k: per_kernel[k]["ms_total"]) if graded else None

    # ---- seeded evaluation key: b halves on the device, a halves regenerated ----
    seeded = None
    if not args.no_rotate:
        evk_b_t = g.to_device(g.he_keygen_seeded(ctx, ks + 1000 * rank + 3, sk), dev)
        g.he_evk_register_seeded(ctx, evk_b_t, ks + 1000 * rank + 3)
        for k in range(3):
            a, b = ct_t[k % NPAIRS]
            g.he_mul_rescale(ctx, a, b, evk_b_t, level, outs[k % NPAIRS], ws, stream)
        torch.cuda.synchronize()
        zs = g.he_decrypt(ctx, sk, g.to_host(outs[2]), level - 1, sc * sc / float(ctx.q[level - 1]))
        m_s = si.messages(N // 2, s1 + 34) * si.messages(N // 2, s2 + 34)
        reps = max(20, min(args.steps, 1000))
        s0e, s1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0e.record(stream)
        for k in range(reps):
            a, b = ct_t[k % NPAIRS]
            g.he_mul_rescale(ctx, a, b, evk_b_t, level, outs[k % NPAIRS], ws, stream)
        s1e.record(stream)
        torch.cuda.synchronize()
        sms = s0e.elapsed_time(s1e) / reps
        g.he_profile(ctx, True)
        for k in range(20):
            a, b = ct_t[k % NPAIRS]
            g.he_mul_rescale(ctx, a, b, evk_b_t, level, outs[k % NPAIRS], ws, stream)
        sprof = g.he_profile_read(ctx)
        g.he_profile(ctx, False)
        ip = sprof.get("inner_product")
        seeded = {"HE_Mul_per_s": 1e3 / sms, "ms": sms, "reps": reps,
                  "evk_bytes": int(evk_b_t.numel() * 8), "evk_bytes_unseeded": int(evk_t.numel() * 8),
                  "inner_product_us": (ip[0] / ip[1] * 1e3) if ip else None,
                  "decrypt_max_err": float(np.abs(zs - m_s).max())}
        g.he_evk_unregister(ctx, evk_b_t)
        del evk_b_t

    # ---- ModDown and rescale as one division by P q_{l-1} (different words) ----
    pq = None
    if not args.no_rotate:
        for k in range(3):
            a, b = ct_t[k % NPAIRS]
            g.he_mul_rescale_pq(ctx, a, b, evk_t, level, outs[k % NPAIRS], ws, stream)
        torch.cuda.synchronize()
        zq = g.he_decrypt(ctx, sk, g.to_host(outs[2]), level - 1, sc * sc / float(ctx.q[level - 1]))
        m_q = si.messages(N // 2, s1 + 34) * si.messages(N // 2, s2 + 34)
        reps = max(20, min(args.steps, 1000))
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        for k in range(reps):
            a, b = ct_t[k % NPAIRS]
            g.he_mul_rescale_pq(ctx, a, b, evk_t, level, outs[k % NPAIRS], ws, stream)
        q1.record(stream)
        torch.cuda.synchronize()
        qms = q0.elapsed_time(q1) / reps
        g.he_profile(ctx, True)
        for k in range(20):
            a, b = ct_t[k % NPAIRS]
            g.he_mul_rescale_pq(ctx, a, b, evk_t, level, outs[k % NPAIRS], ws, stream)
        qprof = g.he_profile_read(ctx)
        g.he_profile(ctx, False)
        md = qprof.get("moddown_conv")
        pq = {"HE_Mul_per_s": 1e3 / qms, "ms": qms, "reps": reps,
              "moddown_conv_us": (md[0] / md[1] * 1e3) if md else None,
              "decrypt_max_err": float(np.abs(zq - m_q).max())}

    # ---- HE rotation (Galois automorphism + key switch) on the same workload ----
    rot = None
    if not args.no_rotate:
        gal = g.he_galois_elt(ctx, 1)
        rk_t = g.to_device(g.he_keygen_rot(ctx, ks + 77, sk, gal), dev)
        rot_out = torch.empty((2, level, N), dtype=torch.int64, device=dev)
        for k in range(3):
            g.he_rotate(ctx, ct_t[k % NPAIRS][0], rk_t, level, gal, rot_out, ws, stream)
        torch.cuda.synchronize()
        zr = g.he_decrypt(ctx, sk, g.to_host(rot_out), level, sc)
        rot_err = float(np.abs(zr - np.roll(si.messages(N // 2, s1 + 17 * 2), -1)).max())
        reps = max(20, min(args.steps, 1000))
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r0.record(stream)
        for k in range(reps):
            g.he_rotate(ctx, ct_t[k % NPAIRS][0], rk_t, level, gal, rot_out, ws, stream)
        r1.record(stream)
        torch.cuda.synchronize()
        rms = r0.elapsed_time(r1) / reps
        rot = {"HE_Rotate_per_s": 1e3 / rms, "ms": rms, "level": level, "steps": 1, "reps": reps,
               "decrypt_max_err": rot_err}
        del rk_t

    # ---- a multiplication chain down the levels (HE Mul + rescale at every level) ----
    chain = None
    if not args.no_rotate and level > 2:
        outs_c = [torch.empty((2, l - 1, N), dtype=torch.int64, device=dev) for l in range(level, 1, -1)]

        def run_chain():
            cur = ct_t[0][0]
            for k, l in enumerate(range(level, 1, -1)):
                g.he_mul_rescale(ctx, cur, cur, evk_t, l, outs_c[k], ws, stream)
                cur = outs_c[k]

        for _ in range(3):
            run_chain()
        torch.cuda.synchronize()
        creps = 20
        c0, c1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _ in range(creps):
            run_chain()
        c1e.record(stream)
        torch.cuda.synchronize()
        cms = c0.elapsed_time(c1e) / creps
        chain = {"levels": f"{level}->1", "he_muls": level - 1, "ms_per_chain": cms,
                 "HE_Mul_per_s": (level - 1) / (cms * 1e-3), "reps": creps}

    # ---- the paper's own non-RNS HE Mul at its parameters (N=2^16, log Q=1200, log p=30) ----
    nonrns = None
    if not args.no_rotate and preset == "n16":
        nr_ctx = g.Context(g.Params(16, 64, 1, 16, 57, 57, 192), device=True)
        plan = g.NrPlan(nr_ctx, 1200, 30)
        NW = (1200 + 63) // 64

        def words(k, seed):  # a seeded BigInt polynomial mod 2^k, word-major
            a = si.uniform_residues([1 << 62] * ((k + 63) // 64), (N,), seed)
            a = (a << np.uint64(2)) | (a & np.uint64(3))
            if k % 64:
                a[-1] &= np.uint64((1 << (k % 64)) - 1)
            return a

        nct = [(g.to_device(np.stack([words(1200, 11000 + 4 * k), words(1200, 11001 + 4 * k)]), dev),
                g.to_device(np.stack([words(1200, 11002 + 4 * k), words(1200, 11003 + 4 * k)]), dev)) for k in range(2)]
        nevk = g.to_device(np.stack([words(2400, 11100), words(2400, 11101)]), dev)
        prep = plan.prepare_evk(nevk, stream)
        nws = plan.workspace(device=dev)
        nout = torch.empty((2, NW, N), dtype=torch.int64, device=dev)
        for k in range(3):
            plan.mul(nct[k % 2][0], nct[k % 2][1], prep, 1200, nout, nws, stream)
        torch.cuda.synchronize()
        nreps = 30
        n0, n1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n0.record(stream)
        for k in range(nreps):
            plan.mul(nct[k % 2][0], nct[k % 2][1], prep, 1200, nout, nws, stream)
        n1.record(stream)
        torch.cuda.synchronize()
        nms = n0.elapsed_time(n1) / nreps
        g.he_profile(nr_ctx, True)
        for k in range(10):
            plan.mul(nct[k % 2][0], nct[k % 2][1], prep, 1200, nout, nws, stream)
        nprof = g.he_profile_read(nr_ctx)
        g.he_profile(nr_ctx, False)
        nonrns = {"workload": "the paper's non-RNS HEAAN HE Mul (Fig. 2): N=2^16, log Q=1200 (19-word BigInts), "
                              f"CRT to {plan.np1}/{plan.np2} 57-bit primes, evk mod Q^2",
                  "ms_per_he_mul": nms, "HE_Mul_per_s": 1e3 / nms, "reps": nreps,
                  "paper_gpu_ms": 38.1, "paper_gpu": "Titan RTX, GPU-CLH, 32-bit words (context, other hardware)",
                  "kernels_us": {k: v[0] / v[1] * 1e3 for k, v in nprof.items()},
                  "data": "seeded uniform words (same work as encryptions)"}
        plan.close()
        del nws, prep, nevk, nct, nout

    # ALU ceilings: the NTT's butterfly and the conversions' inner loop,
    # register-resident, measured in this run at its clocks
    bfly_peak = g.he_probe_butterfly_rate(152 * 8, 4096, stream)
    conv_width = {"modup": kernel_width(prm.alpha), "moddown_conv": kernel_width(prm.K)}
    conv_peak = {k: g.he_probe_conversion_rate(w, 152 * 8, max(64, 4096 // w), stream) for k, w in conv_width.items()}
    probe = {"butterfly_per_s": bfly_peak, "conversion_mac_per_s": conv_peak, "conversion_width": conv_width}
    # the CUDA-core remainder of a byte-split tensor-core conversion (planes ->
    # 128 bits -> reduction) against the whole CUDA-core conversion, per output
    recomb = g.he_probe_recombine_rate(152 * 8, 1024, stream)
    probe["byte_split_tensor_conversion"] = {
        "recombine_outputs_per_s": recomb,
        "cuda_core_outputs_per_s": {k: conv_peak[k] / w for k, w in conv_width.items()},
        "what": "outputs/s of the CUDA-core work left per output by a byte-split tensor-core conversion (13 fp32 "
                "planes to 128 bits, lazy Barrett; MMA not counted) beside the outputs/s of the whole CUDA-core "
                "conversion at the kernels' widths: below 1 means the tensor-core form cannot be faster"}
    probe["byte_split_tensor_conversion"]["ratio"] = {
        k: recomb / v for k, v in probe["byte_split_tensor_conversion"]["cuda_core_outputs_per_s"].items()}
    for k, d in per_kernel.items():
        if d["kind"] == "alu":
            d["frac_of_probe"] = d["Gbutterfly_s"] * 1e9 / bfly_peak
        elif d["kind"] == "mac" and k.split(".")[0] in conv_peak:
            d["frac_of_probe"] = d["GMAC_s"] * 1e9 / conv_peak[k.split(".")[0]]
        elif d["kind"] == "mixed":
            # the ModDown conversion (ALU) and the q rows' key-switch sums (HBM)
            # in one launch: each part's rate, and the launch against the two
            # ideal times added (the bound if the parts did not overlap)
            macs = kernel_work(k, ctx.prm, level, split)[1]
            beta = -(-level // ctx.prm.alpha)
            qbytes = (3 * beta + 2) * (level - 1) * ctx.N * 8
            t = d["ms_avg"] * 1e-3
            d["GMAC_s"] = macs / t / 1e9
            d["GB_s"] = qbytes / t / 1e9
            d["frac_of_serial_bound"] = (macs / conv_peak["moddown_conv"] + qbytes / (hbm_peak_gbs() * 1e9)) / t
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    roof = None
    if dom:
        kind, work = kernel_work(dom, ctx.prm, level, split)
        avg_s = per_kernel[dom]["ms_avg"] * 1e-3
        if kind == "alu":
            ach = work / avg_s / 1e9
            roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": bfly_peak / 1e9,
                    "unit": "Gbutterfly/s", "frac": ach / (bfly_peak / 1e9), "traffic": committed_traffic(dom),
                    "peak_source": "measured: the NTT's own butterfly on register-resident data "
                                   "(he_probe_butterfly_rate), same clocks, same run"}
        elif kind == "mac":
            ach = work / avg_s / 1e9
            pk = conv_peak[dom.split(".")[0]] / 1e9
            roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": pk,
                    "unit": "GMAC/s", "frac": ach / pk, "traffic": committed_traffic(dom),
                    "peak_source": f"measured: the conversion's own inner loop (split-28 Karatsuba multiply-"
                                   f"accumulates, reduction from the accumulators) at width {conv_width[dom.split('.')[0]]}, "
                                   f"register-resident (he_probe_conversion_rate), same clocks, same run"}
        elif kind == "hbm":
            ach = work / avg_s / 1e9
            roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                    "frac": ach / hbm_peak, "traffic": committed_traffic(dom),
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs"}
    # HBM view of the key-switch inner product (the evk stream)
    ip = inner_product_alone(g, ctx, step, level)

    # ---- the same single HE Mul at N = 2^17 (level 44 -> 43, dnum 4) ----
    n17 = None
    if preset == "n16" and not args.no_n17:
        n17 = run_single(g, "n17", WORKLOADS["n17"][1], dev, stream, rank)

    # ---- batched configuration: 64 HE Muls at uneven levels, one launch sequence ----
    batched = None
    if preset == "n16" and not args.no_batch:
        batched = run_batched(g, ctx, evk_t, dev, stream, wsz)

    serving = None
    if preset == "n16" and not args.no_serve:
        serving = {"poisson_2000": run_serving(g, dev),
                   "saturating_20000": run_serving(g, dev, rate_hz=20000.0, duration_s=2.0)}

    # ---- CPU oracle baseline (rank 0, N=1 only) ----
    cpu = None
    if rank == 0 and wsz == 1 and not args.no_cpu_baseline:
        budget = float(os.environ.get("HE_CPU_BUDGET_S", "20"))
        cores = host_cores()
        agg, done, rates = time_oracle_cores(preset, level, budget, cores)
        cpu = {"value": agg, "unit": "HE Mul/s", "cores": cores, "kind": "oracle",
               "sample": f"{done} full HE Mul+rescale runs of the plain single-threaded oracle at the same "
                         f"workload, one process per host core ({cores}), ~{budget:.0f} s each",
               "single_core_value": min(rates)}

    if rank == 0:
        line = {
            "metric": "HE Mul/s (HE Mul + relinearize + rescale)", "value": value, "unit": "HE Mul/s",
            "n_gpus": wsz, "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic: seeded encryptions of unit-disk messages, seeded keys",
            "config": {"workload": desc, "N": N, "level": level, "L": prm.L, "K": prm.K, "alpha": prm.alpha,
                       "dnum": ctx.dnum, "l2": f"{NPAIRS} distinct ciphertext pairs + evk rotated "
                       f"({(NPAIRS * 4 * level + 2 * ctx.dnum * (prm.K + prm.L)) * N * 8 / 1e6:.0f} MB > 129 MB L2)",
                       "parallelism": f"replicas x{wsz}"},
            "repeats": {"regions": len(rep_ms), "steps_each": args.steps,
                        "value_median": job_rate(args.steps, wsz, float(np.median(rep_ms)) * 1e-3),
                        "values": [job_rate(args.steps, wsz, m * 1e-3) for m in rep_ms]},
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "mean": float(lat.mean()), "steps": lat_steps},
            "e2e": {"value": e2e_val, "unit": "HE Mul/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "api": f"he_mul_rescale_host_stream, {e2e_steps} steps from pinned host buffers, {slots} slots, "
                           f"median of {len(e2e_runs)} runs",
                    "runs": e2e_runs,
                    "link": {"value": link_val, "unit": "HE Mul/s",
                             "what": "the same bytes per step as plain pinned-host copies (the two uploads and the "
                                     "download each on its own stream), no kernels"},
                    "decrypt_max_err": e2e_err,
                    "single_call": {"value": single_val, "unit": "HE Mul/s", "api": "he_mul_rescale_host",
                                    "steps": single_steps}},
            "gpu_launches": launches_per_step * args.steps,
            "roofline": roof,
            "inner_product_hbm": ip,
            "probe": probe,
            "kernels": per_kernel,
            "autotune": dict(shape_dict(tune_best), tried=[shape_dict(t) for t in tune_tried]),
            "n17_single": n17,
            "rescale_pq": pq,
            "seeded_evk": seeded,
            "nonrns_paper": nonrns,
            "rotate": rot,
            "chain": chain,
            "batched": batched,
            "serving": serving,
            "cpu_baseline": cpu,
            "clocks": clk,
            "decrypt_max_err": dec_err,
        }
        print(json.dumps(line), flush=True)
    if wsz > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="n16", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-rotate", action="store_true")
    ap.add_argument("--no-n17", action="store_true", help="skip the N=2^17 single HE Mul section")
    ap.add_argument("--shape", default="", help="fixed launch shape CAP,CHUNK,PDL[,R8[,IPJOBS[,FUSE[,SPLIT[,SMALL"
                                                 "[,ONEPASS]]]]]] "
                                                 "instead of autotuning")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
