"""CKKS encoding / decoding for the oracle (TEST INFRASTRUCTURE ONLY).

Sec. 3.1 of the paper: a message of n <= N/2 complex numbers is scaled by Delta
and turned into an integer polynomial of Z[X]/(X^N + 1).  The paper defers the
map itself to the HEAAN paper; the reading used here is the canonical
embedding with full packing (n = N/2): slot k holds t(zeta^(5^k mod 2N)) with
zeta = exp(i*pi/N), and slot k's conjugate sits at the root zeta^(-5^k).

The paper says the scaled values are "rounded down"; the reading here rounds
to the nearest integer (np.rint), which the usual CKKS error bound assumes.
numpy's FFT is used as a library primitive for the evaluation at all odd
powers of zeta:
    t(zeta^(2r+1)) = sum_j (t_j zeta^j) exp(2 pi i r j / N) = N * ifft(t * zeta^j)[r].
"""
from __future__ import annotations

import numpy as np


def slot_rows(logN: int) -> tuple[np.ndarray, np.ndarray]:
    """r indices of the odd powers zeta^(2r+1) that hold slot k and its conjugate."""
    N = 1 << logN
    twoN = 2 * N
    e = np.empty(N // 2, dtype=np.int64)
    x = 1
    for k in range(N // 2):
        e[k] = x
        x = (x * 5) % twoN
    rows = (e - 1) // 2
    conj = (twoN - e - 1) // 2
    return rows, conj


def _zeta_pow(logN: int, sign: int) -> np.ndarray:
    N = 1 << logN
    j = np.arange(N)
    return np.exp(sign * 1j * np.pi * j / N)


def decode(coeffs: np.ndarray, logN: int) -> np.ndarray:
    """Evaluate the (already 1/Delta-scaled) real polynomial at the slot roots."""
    N = 1 << logN
    v = np.fft.ifft(np.asarray(coeffs, dtype=np.float64) * _zeta_pow(logN, +1)) * N
    rows, _ = slot_rows(logN)
    return v[rows]


def encode_float(z: np.ndarray, logN: int, delta: float) -> np.ndarray:
    """Real coefficients t_j of the polynomial whose slot values are delta*z (no rounding)."""
    N = 1 << logN
    z = np.asarray(z, dtype=np.complex128)
    assert z.shape == (N // 2,)
    rows, conj = slot_rows(logN)
    full = np.zeros(N, dtype=np.complex128)
    full[rows] = delta * z
    full[conj] = np.conj(delta * z)
    # t_j = (1/N) sum_r full[r] zeta^-(2r+1)j = zeta^-j * fft(full)[j] / N
    t = np.fft.fft(full) * _zeta_pow(logN, -1) / N
    return t.real


def encode(z: np.ndarray, logN: int, delta: float) -> np.ndarray:
    """Integer plaintext coefficients (int64), rounded to nearest."""
    return np.rint(encode_float(z, logN, delta)).astype(np.int64)
