"""Seeded synthetic inputs shared by the tests, the oracle and the benchmark.

This module holds none of the method's arithmetic: it only draws the values a
user would hand to the library (complex messages, per-item levels of a batch,
request arrival times and mixes, raw residues for throughput runs).  Every draw
is a numpy ``Generator(PCG64(seed))`` so both sides of a comparison receive
identical inputs.

Distributions (the paper uses synthetic complex messages, Sec. 2 / Sec. 3.1):
  * messages: n complex numbers uniform in the unit disk, r = sqrt(U), theta = 2 pi U'
  * batch levels: integers uniform in [lo, hi]
  * serving: Poisson arrivals (exponential gaps) with a two-class mix
"""
from __future__ import annotations

import numpy as np

# Seeds fixed per workload (keys, message 1, message 2).
SEEDS = {
    "n12": (1201, 1202, 1203),
    "n15": (1501, 1502, 1503),
    "n16": (1601, 1602, 1603),
    "n17": (1701, 1702, 1703),
}
BATCH_SEED = 1604
SERVE_SEED = 1501


def messages(n: int, seed: int) -> np.ndarray:
    """n complex values uniform in the unit disk."""
    g = np.random.Generator(np.random.PCG64(seed))
    r = np.sqrt(g.random(n))
    th = 2.0 * np.pi * g.random(n)
    return r * np.cos(th) + 1j * r * np.sin(th)


def batch_levels(count: int, lo: int, hi: int, seed: int = BATCH_SEED) -> np.ndarray:
    """Per-item levels (limb counts) uniform in [lo, hi]."""
    g = np.random.Generator(np.random.PCG64(seed))
    return g.integers(lo, hi + 1, size=count).astype(np.int64)


def uniform_residues(moduli, shape_tail: tuple[int, ...], seed: int) -> np.ndarray:
    """Array [len(moduli), *shape_tail] with row i uniform in [0, moduli[i])."""
    g = np.random.Generator(np.random.PCG64(seed))
    rows = [g.integers(0, int(m), size=shape_tail, dtype=np.uint64) for m in moduli]
    return np.stack(rows, axis=0)


def poisson_arrivals(rate_hz: float, duration_s: float, seed: int = SERVE_SEED) -> np.ndarray:
    """Arrival times (seconds) of a Poisson stream of the given rate."""
    g = np.random.Generator(np.random.PCG64(seed))
    n_max = int(rate_hz * duration_s * 1.5) + 64
    gaps = g.exponential(1.0 / rate_hz, size=n_max)
    t = np.cumsum(gaps)
    return t[t < duration_s]


def serving_mix(n: int, seed: int = SERVE_SEED + 1,
                classes=((0.7, 15, 2, 16), (0.3, 16, 4, 24))) -> list[tuple[int, int]]:
    """(logN, level) per request: each class is (probability, logN, level_lo, level_hi)."""
    g = np.random.Generator(np.random.PCG64(seed))
    probs = np.array([c[0] for c in classes])
    which = g.choice(len(classes), size=n, p=probs / probs.sum())
    out = []
    for w in which:
        _, logN, lo, hi = classes[w]
        out.append((logN, int(g.integers(lo, hi + 1))))
    return out
