"""Python binding of the GB300 full-RNS CKKS HE Mul library (libhe_gb300.so).

Argument marshalling only: every step of HE Mul runs in the library's CUDA
kernels.  Device buffers are torch tensors (int64 storage holding the uint64
residues, which are all below 2^57); streams are torch streams.  Host arrays
are numpy.  Function names mirror the C ABI in include/he.h.

There is no CPU fallback: if the compiled library is missing, importing the
device entry points raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhe_gb300.so")

HE_OK, HE_EINVAL, HE_ELEVEL, HE_ENOMEM, HE_ECUDA, HE_ETIMEOUT, HE_EBUSY = range(7)


class HeError(RuntimeError):
    def __init__(self, code: int, what: str):
        msg = f"{what}: {lib().he_strerror(code).decode()} (code {code})"
        if code == HE_ECUDA:
            msg += f" [{lib().he_last_cuda_error().decode()}]"
        super().__init__(msg)
        self.code = code


class he_params(ctypes.Structure):
    _fields_ = [("logN", ctypes.c_int), ("L", ctypes.c_int), ("K", ctypes.c_int), ("alpha", ctypes.c_int),
                ("q_bits", ctypes.c_int), ("p_bits", ctypes.c_int), ("h", ctypes.c_int),
                ("sigma", ctypes.c_double)]


class he_request(ctypes.Structure):
    _fields_ = [("ctx_index", ctypes.c_int), ("level", ctypes.c_int), ("ct1", ctypes.c_void_p),
                ("ct2", ctypes.c_void_p), ("out", ctypes.c_void_p), ("ready", ctypes.c_void_p)]


class he_server_report(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("pending", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("mean_batch", ctypes.c_double), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("throughput", ctypes.c_double)]


class he_job(ctypes.Structure):
    _fields_ = [("ct1", ctypes.c_void_p), ("ct2", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("level", ctypes.c_int)]


_lib = None

_SIGS = {
    "he_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "he_last_cuda_error": (ctypes.c_char_p, []),
    "he_ctx_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "he_ctx_create_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "he_ctx_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "he_ctx_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "he_keygen": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p]),
    "he_keygen_from_sk": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p]),
    "he_encode": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                 ctypes.c_double, ctypes.c_void_p]),
    "he_decode": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_size_t]),
    "he_encrypt_poly": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                       ctypes.c_uint64, ctypes.c_void_p]),
    "he_encrypt": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_size_t, ctypes.c_double, ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p]),
    "he_decrypt_poly": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                       ctypes.c_void_p]),
    "he_decrypt": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "he_evk_upload": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "he_workspace_bytes": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int]),
    "he_mul": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "he_mul_rescale": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                      ctypes.c_void_p]),
    "he_mul_rescale_pq": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                      ctypes.c_void_p]),
    "he_rescale": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_size_t, ctypes.c_void_p]),
    "he_step_ntt": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_void_p]),
    "he_step_tensor": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                      ctypes.c_void_p, ctypes.c_void_p]),
    "he_step_modup": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "he_step_inner_product": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                             ctypes.c_void_p]),
    "he_step_moddown": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "he_batch_workspace_bytes": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "he_host_workspace_bytes": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int]),
    "he_mul_rescale_static": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "he_mul_rescale_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                           ctypes.c_void_p]),
    "he_host_stream_workspace_bytes": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "he_mul_rescale_host_stream": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                  ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p]),
    "he_profile": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "he_server_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.c_size_t, ctypes.c_int, ctypes.c_int]),
    "he_server_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "he_server_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]),
    "he_server_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int]),
    "he_server_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "he_server_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "he_batch_graph_workspace_bytes": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int]),
    "he_batch_graph_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p]),
    "he_batch_graph_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "he_batch_graph_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "he_probe_butterfly_rate": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "he_probe_conversion_rate": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                                ctypes.c_void_p]),
    "he_probe_recombine_rate": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "he_galois_elt": (ctypes.c_uint64, [ctypes.c_void_p, ctypes.c_int]),
    "he_conj_elt": (ctypes.c_uint64, [ctypes.c_void_p]),
    "he_nr_plan_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "he_nr_plan_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "he_nr_plan_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "he_nr_workspace_bytes": (ctypes.c_size_t, [ctypes.c_void_p]),
    "he_nr_evk_bytes": (ctypes.c_size_t, [ctypes.c_void_p]),
    "he_nr_evk_prepare": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "he_nr_mul": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "he_nr_rescale": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                     ctypes.c_void_p]),
    "he_keygen_seeded": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]),
    "he_evk_register_seeded": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64]),
    "he_evk_unregister": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "he_set_shape": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "he_get_shape": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "he_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_int, ctypes.c_void_p]),
    "he_add": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                              ctypes.c_void_p]),
    "he_sub": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                              ctypes.c_void_p]),
    "he_plain_ntt": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "he_mul_plain": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                    ctypes.c_void_p]),
    "he_add_plain": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                    ctypes.c_void_p]),
    "he_keygen_rot": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint64,
                                     ctypes.c_void_p]),
    "he_rotate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "he_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "he_mul_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
}


def lib():
    """Load libhe_gb300.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_2003_04510_gb300.build.build() first")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != HE_OK:
        raise HeError(rc, what)


def _np_ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _dev_ptr(t) -> int:
    assert t.is_cuda and t.is_contiguous()
    return t.data_ptr()


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


@dataclass
class Params:
    logN: int
    L: int
    K: int
    alpha: int
    q_bits: int
    p_bits: int
    h: int = 64
    sigma: float = 3.2

    def c(self) -> he_params:
        return he_params(self.logN, self.L, self.K, self.alpha, self.q_bits, self.p_bits, self.h, self.sigma)


# Workload presets (ring degree, limb counts, prime sizes, secret weight, scale).
PRESETS = {
    "n12": (Params(12, 3, 1, 1, 50, 51, 64), 40),
    "n15": (Params(15, 16, 8, 8, 54, 55, 192), 50),
    "n16": (Params(16, 24, 8, 8, 54, 55, 192), 50),
    "n17": (Params(17, 44, 12, 11, 54, 54, 192), 50),
}


class Context:
    """Owns an he_ctx*.  device=False builds a host-only context (no CUDA)."""

    def __init__(self, prm: Params, device: bool = True):
        self.prm = prm
        self.ptr = ctypes.c_void_p()
        cp = prm.c()
        fn = lib().he_ctx_create if device else lib().he_ctx_create_host
        _check(fn(ctypes.byref(self.ptr), ctypes.byref(cp)), "he_ctx_create")
        N = ctypes.c_int()
        dnum = ctypes.c_int()
        mod = np.zeros(prm.K + prm.L, dtype=np.uint64)
        _check(lib().he_ctx_info(self.ptr, ctypes.byref(N), ctypes.byref(dnum), _np_ptr(mod)), "he_ctx_info")
        self.N, self.dnum, self.moduli = N.value, dnum.value, mod
        self.device = device

    @property
    def q(self) -> np.ndarray:
        return self.moduli[self.prm.K:]

    @property
    def p(self) -> np.ndarray:
        return self.moduli[: self.prm.K]

    def beta(self, level: int) -> int:
        return -(-level // self.prm.alpha)

    def close(self):
        if self.ptr:
            lib().he_ctx_destroy(self.ptr)
            self.ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- host side --------------------------------------------------------------
def he_keygen(ctx: Context, seed: int):
    N, L, K = ctx.N, ctx.prm.L, ctx.prm.K
    sk = np.zeros(N, dtype=np.int64)
    pk = np.zeros((2, L, N), dtype=np.uint64)
    evk = np.zeros((ctx.dnum, 2, K + L, N), dtype=np.uint64)
    _check(lib().he_keygen(ctx.ptr, seed, _np_ptr(sk), _np_ptr(pk), _np_ptr(evk)), "he_keygen")
    return sk, pk, evk


def he_encode(ctx: Context, z: np.ndarray, scale: float) -> np.ndarray:
    re = np.ascontiguousarray(z.real, dtype=np.float64)
    im = np.ascontiguousarray(z.imag, dtype=np.float64)
    out = np.zeros(ctx.N, dtype=np.int64)
    _check(lib().he_encode(ctx.ptr, _np_ptr(re), _np_ptr(im), len(re), scale, _np_ptr(out)), "he_encode")
    return out


def he_decode(ctx: Context, coeffs: np.ndarray) -> np.ndarray:
    c = np.ascontiguousarray(coeffs, dtype=np.float64)
    re = np.zeros(ctx.N // 2)
    im = np.zeros(ctx.N // 2)
    _check(lib().he_decode(ctx.ptr, _np_ptr(c), _np_ptr(re), _np_ptr(im), ctx.N // 2), "he_decode")
    return re + 1j * im


def he_encrypt_poly(ctx: Context, pk: np.ndarray, pt: np.ndarray, level: int, seed: int) -> np.ndarray:
    ct = np.zeros((2, level, ctx.N), dtype=np.uint64)
    pt = np.ascontiguousarray(pt, dtype=np.int64)
    _check(lib().he_encrypt_poly(ctx.ptr, _np_ptr(np.ascontiguousarray(pk)), _np_ptr(pt), level, seed, _np_ptr(ct)),
           "he_encrypt_poly")
    return ct


def he_encrypt(ctx: Context, pk: np.ndarray, z: np.ndarray, scale: float, level: int, seed: int) -> np.ndarray:
    re = np.ascontiguousarray(z.real, dtype=np.float64)
    im = np.ascontiguousarray(z.imag, dtype=np.float64)
    ct = np.zeros((2, level, ctx.N), dtype=np.uint64)
    _check(lib().he_encrypt(ctx.ptr, _np_ptr(np.ascontiguousarray(pk)), _np_ptr(re), _np_ptr(im), len(re), scale,
                            level, seed, _np_ptr(ct)), "he_encrypt")
    return ct


def he_decrypt_poly(ctx: Context, sk: np.ndarray, ct: np.ndarray, level: int) -> np.ndarray:
    m = np.zeros((level, ctx.N), dtype=np.uint64)
    _check(lib().he_decrypt_poly(ctx.ptr, _np_ptr(np.ascontiguousarray(sk, dtype=np.int64)),
                                 _np_ptr(np.ascontiguousarray(ct, dtype=np.uint64)), level, _np_ptr(m)),
           "he_decrypt_poly")
    return m


def he_decrypt(ctx: Context, sk: np.ndarray, ct: np.ndarray, level: int, scale: float) -> np.ndarray:
    re = np.zeros(ctx.N // 2)
    im = np.zeros(ctx.N // 2)
    _check(lib().he_decrypt(ctx.ptr, _np_ptr(np.ascontiguousarray(sk, dtype=np.int64)),
                            _np_ptr(np.ascontiguousarray(ct, dtype=np.uint64)), level, scale, _np_ptr(re),
                            _np_ptr(im), ctx.N // 2), "he_decrypt")
    return re + 1j * im


# ---- device side (torch tensors as device buffers) ----------------------------
def to_device(a: np.ndarray, device="cuda"):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).to(device)


def to_host(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def he_workspace_bytes(ctx: Context, level: int) -> int:
    return int(lib().he_workspace_bytes(ctx.ptr, level))


def workspace(ctx: Context, level: int, device="cuda"):
    import torch
    nbytes = he_workspace_bytes(ctx, level)
    return torch.empty(nbytes // 8, dtype=torch.int64, device=device)


def he_mul(ctx, ct1, ct2, evk, level, out, ws, stream=None):
    _check(lib().he_mul(ctx.ptr, _dev_ptr(ct1), _dev_ptr(ct2), _dev_ptr(evk), level, _dev_ptr(out), _dev_ptr(ws),
                        ws.numel() * 8, _stream_ptr(stream)), "he_mul")


def he_mul_rescale(ctx, ct1, ct2, evk, level, out, ws, stream=None):
    _check(lib().he_mul_rescale(ctx.ptr, _dev_ptr(ct1), _dev_ptr(ct2), _dev_ptr(evk), level, _dev_ptr(out),
                                _dev_ptr(ws), ws.numel() * 8, _stream_ptr(stream)), "he_mul_rescale")


def he_mul_rescale_pq(ctx, ct1, ct2, evk, level, out, ws, stream=None):
    """HE Mul with ModDown and rescale as one division by P q_{level-1}."""
    _check(lib().he_mul_rescale_pq(ctx.ptr, _dev_ptr(ct1), _dev_ptr(ct2), _dev_ptr(evk), level, _dev_ptr(out),
                                   _dev_ptr(ws), ws.numel() * 8, _stream_ptr(stream)), "he_mul_rescale_pq")


# he_mul_rescale_static's scratch size (HE_STATIC_SCRATCH_BYTES in he.h)
HE_STATIC_SCRATCH_BYTES = 64 << 20


def he_mul_rescale_static(ctx, ct1, ct2, evk, level, out, stream=None):
    """he_mul_rescale with the library's fixed device scratch as workspace (no allocation)."""
    _check(lib().he_mul_rescale_static(ctx.ptr, _dev_ptr(ct1), _dev_ptr(ct2), _dev_ptr(evk), level, _dev_ptr(out),
                                       _stream_ptr(stream)), "he_mul_rescale_static")


def he_add(ctx, ct1, ct2, level, out, stream=None):
    _check(lib().he_add(ctx.ptr, _dev_ptr(ct1), _dev_ptr(ct2), level, _dev_ptr(out), _stream_ptr(stream)), "he_add")


def he_sub(ctx, ct1, ct2, level, out, stream=None):
    _check(lib().he_sub(ctx.ptr, _dev_ptr(ct1), _dev_ptr(ct2), level, _dev_ptr(out), _stream_ptr(stream)), "he_sub")


def he_plain_ntt(ctx, coeffs: np.ndarray, level: int) -> np.ndarray:
    pt = np.zeros((level, ctx.N), dtype=np.uint64)
    _check(lib().he_plain_ntt(ctx.ptr, _np_ptr(np.ascontiguousarray(coeffs, dtype=np.int64)), level, _np_ptr(pt)),
           "he_plain_ntt")
    return pt


def he_mul_plain(ctx, ct, pt, level, out, stream=None):
    _check(lib().he_mul_plain(ctx.ptr, _dev_ptr(ct), _dev_ptr(pt), level, _dev_ptr(out), _stream_ptr(stream)),
           "he_mul_plain")


def he_add_plain(ctx, ct, pt, level, out, stream=None):
    _check(lib().he_add_plain(ctx.ptr, _dev_ptr(ct), _dev_ptr(pt), level, _dev_ptr(out), _stream_ptr(stream)),
           "he_add_plain")


class he_shape(ctypes.Structure):
    _fields_ = [("group_cap", ctypes.c_int), ("modup_chunk", ctypes.c_int), ("pdl", ctypes.c_int),
                ("ntt_r8", ctypes.c_int), ("ip_jobs", ctypes.c_int), ("fuse", ctypes.c_int), ("ntt_split", ctypes.c_int),
                ("ntt_small", ctypes.c_int), ("ntt_onepass", ctypes.c_int), ("ms", ctypes.c_double)]


def _shape_tuple(sh) -> tuple:
    return (sh.group_cap, sh.modup_chunk, sh.pdl, sh.ntt_r8, sh.ip_jobs, sh.fuse, sh.ntt_split, sh.ntt_small,
            sh.ntt_onepass)


def he_set_shape(ctx, group_cap: int, modup_chunk: int, pdl: int = 1, ntt_r8: int = 0, ip_jobs: int = 8,
                 fuse: int = 7, ntt_split: int = 0, ntt_small: int = 0, ntt_onepass: int = 0):
    sh = he_shape(group_cap, modup_chunk, pdl, ntt_r8, ip_jobs, fuse, ntt_split, ntt_small, ntt_onepass, 0.0)
    _check(lib().he_set_shape(ctx.ptr, ctypes.byref(sh)), "he_set_shape")


def he_get_shape(ctx) -> tuple[int, int, int, int, int, int, int, int, int]:
    """(group_cap, modup_chunk, pdl, ntt_r8, ip_jobs, fuse, ntt_split, ntt_small, ntt_onepass)"""
    sh = he_shape()
    _check(lib().he_get_shape(ctx.ptr, ctypes.byref(sh)), "he_get_shape")
    return _shape_tuple(sh)


def he_autotune(ctx, jobs, evk, ws, reps: int = 3, stream=None):
    """jobs: list of (ct1, ct2, out, level) device tensors (one job: the single
    path).  Returns (best (cap, chunk, pdl, ntt_r8, ip_jobs, fuse, ntt_split,
    ntt_small, ntt_onepass, ms), [the same for every shape tried])."""
    arr = (he_job * len(jobs))()
    for i, (a, b, o, lv) in enumerate(jobs):
        arr[i] = he_job(_dev_ptr(a), _dev_ptr(b), _dev_ptr(o), int(lv))
    best = he_shape()
    tried = (he_shape * 1024)()
    n = ctypes.c_int()
    _check(lib().he_autotune(ctx.ptr, ctypes.cast(arr, ctypes.c_void_p), len(jobs), _dev_ptr(evk), _dev_ptr(ws),
                             ws.numel() * 8, reps, _stream_ptr(stream), ctypes.byref(best),
                             ctypes.cast(tried, ctypes.c_void_p), 1024, ctypes.byref(n)), "he_autotune")
    return (_shape_tuple(best) + (best.ms,), [_shape_tuple(t) + (t.ms,) for t in tried[: n.value]])


def he_keygen_seeded(ctx, seed: int, sk: np.ndarray) -> np.ndarray:
    """b halves [dnum][K+L][N] of the seeded evaluation key of `seed`."""
    prm = ctx.prm
    evk_b = np.zeros((ctx.dnum, prm.K + prm.L, ctx.N), dtype=np.uint64)
    _check(lib().he_keygen_seeded(ctx.ptr, seed, _np_ptr(np.ascontiguousarray(sk, dtype=np.int64)),
                                  _np_ptr(evk_b)), "he_keygen_seeded")
    return evk_b


def he_evk_register_seeded(ctx, evk_b_dev, seed: int):
    _check(lib().he_evk_register_seeded(ctx.ptr, _dev_ptr(evk_b_dev), seed), "he_evk_register_seeded")


def he_evk_unregister(ctx, evk_dev):
    _check(lib().he_evk_unregister(ctx.ptr, _dev_ptr(evk_dev)), "he_evk_unregister")


class NrPlan:
    """The paper's non-RNS HE Mul (BigInt coefficients modulo powers of two) on a
    context created with q_bits = 57 and enough primes (he_nr_plan_*)."""

    def __init__(self, ctx: Context, logQ: int, logp: int):
        self.ctx, self.logQ, self.logp = ctx, logQ, logp
        self.ptr = ctypes.c_void_p()
        _check(lib().he_nr_plan_create(ctx.ptr, logQ, logp, ctypes.byref(self.ptr)), "he_nr_plan_create")
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(lib().he_nr_plan_info(self.ptr, ctypes.byref(a), ctypes.byref(b)), "he_nr_plan_info")
        self.np1, self.np2 = a.value, b.value

    def workspace(self, device="cuda"):
        import torch
        return torch.empty(lib().he_nr_workspace_bytes(self.ptr) // 8, dtype=torch.int64, device=device)

    def prepare_evk(self, evk_dev, stream=None):
        import torch
        prep = torch.empty(lib().he_nr_evk_bytes(self.ptr) // 8, dtype=torch.int64, device=evk_dev.device)
        _check(lib().he_nr_evk_prepare(self.ptr, _dev_ptr(evk_dev), _dev_ptr(prep), _stream_ptr(stream)),
               "he_nr_evk_prepare")
        return prep

    def mul(self, ct1, ct2, prep, logq, out, ws, stream=None):
        _check(lib().he_nr_mul(self.ptr, _dev_ptr(ct1), _dev_ptr(ct2), _dev_ptr(prep), logq, _dev_ptr(out),
                               _dev_ptr(ws), ws.numel() * 8, _stream_ptr(stream)), "he_nr_mul")

    def rescale(self, ct, logq, out, stream=None):
        _check(lib().he_nr_rescale(self.ptr, _dev_ptr(ct), logq, _dev_ptr(out), _stream_ptr(stream)),
               "he_nr_rescale")

    def close(self):
        if self.ptr:
            lib().he_nr_plan_destroy(self.ptr)
            self.ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def he_galois_elt(ctx, steps: int) -> int:
    """5^steps mod 2N (left rotation by `steps` slots)."""
    return int(lib().he_galois_elt(ctx.ptr, int(steps)))


def he_conj_elt(ctx) -> int:
    """2N - 1 (slot-wise complex conjugation)."""
    return int(lib().he_conj_elt(ctx.ptr))


def he_keygen_rot(ctx, seed: int, sk: np.ndarray, galois: int) -> np.ndarray:
    prm = ctx.prm
    rk = np.zeros((ctx.dnum, 2, prm.K + prm.L, ctx.N), dtype=np.uint64)
    _check(lib().he_keygen_rot(ctx.ptr, seed, _np_ptr(np.ascontiguousarray(sk, dtype=np.int64)), galois, _np_ptr(rk)),
           "he_keygen_rot")
    return rk


def he_rotate(ctx, ct, rk, level, galois, out, ws, stream=None):
    _check(lib().he_rotate(ctx.ptr, _dev_ptr(ct), _dev_ptr(rk), level, galois, _dev_ptr(out), _dev_ptr(ws),
                           ws.numel() * 8, _stream_ptr(stream)), "he_rotate")


def he_rescale(ctx, ct, level, out, ws, stream=None):
    _check(lib().he_rescale(ctx.ptr, _dev_ptr(ct), level, _dev_ptr(out), _dev_ptr(ws), ws.numel() * 8,
                            _stream_ptr(stream)), "he_rescale")


def he_step_ntt(ctx, data, prime_idx, inverse: bool, stream=None):
    pi = np.ascontiguousarray(prime_idx, dtype=np.int32)
    _check(lib().he_step_ntt(ctx.ptr, _dev_ptr(data), _np_ptr(pi), len(pi), int(inverse), _stream_ptr(stream)),
           "he_step_ntt")


def he_step_tensor(ctx, ct1, ct2, level, d, stream=None):
    _check(lib().he_step_tensor(ctx.ptr, _dev_ptr(ct1), _dev_ptr(ct2), level, _dev_ptr(d), _stream_ptr(stream)),
           "he_step_tensor")


def he_step_modup(ctx, d2, level, U, ws, stream=None):
    _check(lib().he_step_modup(ctx.ptr, _dev_ptr(d2), level, _dev_ptr(U), _dev_ptr(ws), ws.numel() * 8,
                               _stream_ptr(stream)), "he_step_modup")


def he_step_inner_product(ctx, U, d2, evk, level, KS, ws, stream=None):
    _check(lib().he_step_inner_product(ctx.ptr, _dev_ptr(U), _dev_ptr(d2), _dev_ptr(evk), level, _dev_ptr(KS),
                                       _dev_ptr(ws), ws.numel() * 8, _stream_ptr(stream)), "he_step_inner_product")


def he_step_moddown(ctx, X, level, out, ws, stream=None):
    _check(lib().he_step_moddown(ctx.ptr, _dev_ptr(X), level, _dev_ptr(out), _dev_ptr(ws), ws.numel() * 8,
                                 _stream_ptr(stream)), "he_step_moddown")


def he_batch_workspace_bytes(ctx, levels) -> int:
    lv = np.ascontiguousarray(levels, dtype=np.int32)
    return int(lib().he_batch_workspace_bytes(ctx.ptr, len(lv), _np_ptr(lv)))


def he_mul_batch(ctx, jobs, evk, ws, stream=None):
    """jobs: list of (ct1, ct2, out, level) with device tensors."""
    arr = (he_job * len(jobs))()
    for i, (a, b, o, lv) in enumerate(jobs):
        arr[i] = he_job(_dev_ptr(a), _dev_ptr(b), _dev_ptr(o), int(lv))
    _check(lib().he_mul_batch(ctx.ptr, len(jobs), ctypes.cast(arr, ctypes.c_void_p), _dev_ptr(evk), _dev_ptr(ws),
                              ws.numel() * 8, _stream_ptr(stream)), "he_mul_batch")


def he_host_workspace_bytes(ctx, level) -> int:
    return int(lib().he_host_workspace_bytes(ctx.ptr, level))


def he_mul_rescale_host(ctx, ct1: np.ndarray, ct2: np.ndarray, evk, level, out: np.ndarray, ws, stream=None):
    """ct1, ct2, out: host numpy uint64 arrays (pinned memory gives async copies)."""
    _check(lib().he_mul_rescale_host(ctx.ptr, _np_ptr(ct1), _np_ptr(ct2), _dev_ptr(evk), level, _np_ptr(out),
                                     _dev_ptr(ws), ws.numel() * 8, _stream_ptr(stream)), "he_mul_rescale_host")


def he_host_stream_workspace_bytes(ctx, max_level: int, slots: int = 2) -> int:
    return int(lib().he_host_stream_workspace_bytes(ctx.ptr, max_level, slots))


def he_mul_rescale_host_stream(ctx, ct1s, ct2s, levels, outs, evk, ws, slots: int = 2, stream=None):
    """Jobs from host buffers, pipelined: ct1s[k], ct2s[k] ([2][levels[k]][N])
    and outs[k] ([2][levels[k]-1][N]) are host numpy uint64 arrays (pinned
    memory lets the copies overlap the kernels)."""
    n = len(levels)
    if not (len(ct1s) == len(ct2s) == len(outs) == n):
        raise ValueError("ct1s, ct2s, levels and outs differ in length")
    for a in list(ct1s) + list(ct2s) + list(outs):
        if a.dtype != np.uint64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host buffers must be C-contiguous uint64 arrays")
    p1 = (ctypes.c_void_p * max(n, 1))(*[a.ctypes.data for a in ct1s])
    p2 = (ctypes.c_void_p * max(n, 1))(*[a.ctypes.data for a in ct2s])
    po = (ctypes.c_void_p * max(n, 1))(*[a.ctypes.data for a in outs])
    lv = (ctypes.c_int * max(n, 1))(*[int(v) for v in levels])
    _check(lib().he_mul_rescale_host_stream(ctx.ptr, n, ctypes.cast(p1, ctypes.c_void_p), ctypes.cast(p2, ctypes.c_void_p),
                                            ctypes.cast(lv, ctypes.c_void_p), ctypes.cast(po, ctypes.c_void_p),
                                            _dev_ptr(evk), _dev_ptr(ws), ws.numel() * 8, slots, _stream_ptr(stream)),
           "he_mul_rescale_host_stream")


def he_profile(ctx, enable: bool):
    _check(lib().he_profile(ctx.ptr, int(enable)), "he_profile")


def he_profile_read(ctx, max_kernels: int = 64) -> dict:
    """{kernel name: (total ms, calls)} for the marks recorded since he_profile(ctx, True)."""
    names = ctypes.create_string_buffer(48 * max_kernels)
    ms = np.zeros(max_kernels)
    calls = np.zeros(max_kernels, dtype=np.int32)
    n = ctypes.c_int()
    _check(lib().he_profile_read(ctx.ptr, max_kernels, names, _np_ptr(ms), _np_ptr(calls), ctypes.byref(n)),
           "he_profile_read")
    out = {}
    for j in range(n.value):
        nm = names.raw[48 * j: 48 * j + 48].split(b"\0", 1)[0].decode()
        out[nm] = (float(ms[j]), int(calls[j]))
    return out


def he_probe_butterfly_rate(blocks: int, iters: int, stream=None) -> float:
    r = ctypes.c_double()
    _check(lib().he_probe_butterfly_rate(blocks, iters, ctypes.byref(r), _stream_ptr(stream)),
           "he_probe_butterfly_rate")
    return r.value


def he_probe_conversion_rate(width: int, blocks: int, iters: int, stream=None) -> float:
    r = ctypes.c_double()
    _check(lib().he_probe_conversion_rate(width, blocks, iters, ctypes.byref(r), _stream_ptr(stream)),
           "he_probe_conversion_rate")
    return r.value


def he_probe_recombine_rate(blocks: int, iters: int, stream=None) -> float:
    """Outputs/s of a byte-split tensor-core conversion's CUDA-core remainder
    (13 fp32 planes -> 128 bits -> lazy Barrett), register-resident."""
    r = ctypes.c_double()
    _check(lib().he_probe_recombine_rate(blocks, iters, ctypes.byref(r), _stream_ptr(stream)),
           "he_probe_recombine_rate")
    return r.value


class BatchGraph:
    """he_batch_graph: the batched path captured once in a CUDA graph."""

    def __init__(self, ctx, max_jobs: int, evk, stream=None, device="cuda"):
        import torch
        self.ctx = ctx
        nbytes = int(lib().he_batch_graph_workspace_bytes(ctx.ptr, max_jobs))
        self.ws = torch.empty(nbytes // 8, dtype=torch.int64, device=device)
        self.evk = evk
        self.ptr = ctypes.c_void_p()
        _check(lib().he_batch_graph_create(ctx.ptr, max_jobs, _dev_ptr(evk), _dev_ptr(self.ws), nbytes,
                                           _stream_ptr(stream), ctypes.byref(self.ptr)), "he_batch_graph_create")

    def launch(self, jobs, stream=None):
        arr = (he_job * len(jobs))()
        for i, (a, b, o, lv) in enumerate(jobs):
            arr[i] = he_job(_dev_ptr(a), _dev_ptr(b), _dev_ptr(o), int(lv))
        _check(lib().he_batch_graph_launch(self.ptr, len(jobs), ctypes.cast(arr, ctypes.c_void_p),
                                           _stream_ptr(stream)), "he_batch_graph_launch")

    def close(self):
        if self.ptr:
            lib().he_batch_graph_destroy(self.ptr)
            self.ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """he_server: continuous-batching HE Mul server over several rings."""

    def __init__(self, ctxs, evks, hbm_budget: int, max_batch: int = 64, streams: int = 4):
        n = len(ctxs)
        self._ctxs = (ctypes.c_void_p * n)(*[c.ptr.value for c in ctxs])
        self._evks = (ctypes.c_void_p * n)(*[_dev_ptr(e) for e in evks])
        self._keep = (list(ctxs), list(evks))
        self.ptr = ctypes.c_void_p()
        _check(lib().he_server_create(ctypes.byref(self.ptr), self._ctxs, self._evks, n, hbm_budget, max_batch,
                                      streams), "he_server_create")

    def submit(self, ctx_index: int, level: int, ct1, ct2, out, ready=None) -> int:
        """ready: optional torch.cuda.Event recorded after the operands were written
        (the batch waits for it on the device); None if they are complete."""
        r = he_request(ctx_index, level, _dev_ptr(ct1), _dev_ptr(ct2), _dev_ptr(out),
                       ready.cuda_event if ready is not None else None)
        t = ctypes.c_uint64()
        _check(lib().he_server_submit(self.ptr, ctypes.byref(r), ctypes.byref(t)), "he_server_submit")
        return t.value

    def poll(self, ticket: int) -> bool:
        d = ctypes.c_int()
        _check(lib().he_server_poll(self.ptr, ticket, ctypes.byref(d)), "he_server_poll")
        return bool(d.value)

    def wait(self, ticket: int, timeout_ms: int = 60000):
        _check(lib().he_server_wait(self.ptr, ticket, timeout_ms), "he_server_wait")

    def stats(self) -> dict:
        st = he_server_report()
        _check(lib().he_server_stats(self.ptr, ctypes.byref(st)), "he_server_stats")
        return {f: getattr(st, f) for f, _ in he_server_report._fields_}

    def close(self):
        if self.ptr:
            lib().he_server_destroy(self.ptr)
            self.ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
